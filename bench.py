#!/usr/bin/env python
"""Ray-fan throughput benchmark of the GB300 RTM-GD tracer.

One step = one fan of the anisotropic workload (E + F2 + TID ionosphere on a
91x181x151 FP32 grid, centred dipole, 8/12/16 MHz x 115 elevations x 36
azimuths x O/X = 24,840 rays, RKF45 at rtol 1e-8) traced through the C ABI.
The grid is resident on the device (created once, as in serving); inputs of a
step are the fan arrays.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
                  [--impl ours|reference]

--impl reference times the FP64 CPU oracle on the machine's host cores (a
bounded sample of the same fan per step); it is the baseline arm.
"""
from __future__ import annotations

import argparse
import faulthandler
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "rays/s and ray-steps/s at ≤0.05 km P'/D error; p50/p99 fan latency"

# Algorithmic floating-point operations of one right-hand-side evaluation
# (one RK stage) with the dipole field, counted from the kernel source (an FMA
# counts 2): GD weights 3 x 37 FMA, contraction 192 FMA, grid-coordinate and
# chain factors ~20 flop, dipole + Jacobian ~70, Appleton-Hartree + partials
# ~60, Hamiltonian partials + ray equations ~70, stage offsets and RK
# accumulation ~90 (mixed path; the FP64 path accumulates inside rk*_step64).
FLOP_PER_EVAL = {"mixed": 1000.0, "fp64": 910.0}
# Grid samples one stage evaluation reads: 64 samples (16 rows of 4) plus the
# reference node, FP32 in the mixed path and FP64 in the all-FP64 path.
GATHER_BYTES = {"mixed": 65 * 4, "fp64": 64 * 8}
# DRAM bytes (read + write) of one launch of the benchmark's dominant kernel,
# from an ncu capture of the same launch (cold caches, as after the
# L2 flush between timed steps), keyed by workload and launch configuration
# (kernel, stencil, lanes per ray) and valid only for the kernel sources it
# was captured from: a changed kernel reports traffic null.
KERNEL_SOURCES = ("paper_2506_18579_gb300/csrc/rtgd_kernels.cu", "paper_2506_18579_gb300/csrc/rtgd_device.cuh")
TRAFFIC = {
    # key = (workload, kernel, stencil, lanes per ray); the anisotropic fan in
    # the autotuner's configurations (plain, 4 lanes, 96-thread blocks)
    ("c2", 1, 3, 4): {"bytes_per_launch": 26831616 + 22528, "source_sha256": "2602d2aac951aea9"},
    ("c2", 1, 2, 4): {"bytes_per_launch": 5379072 + 256, "source_sha256": "2602d2aac951aea9"},
    # the ionogram batch, one lane per ray (the only lane count the autotuner
    # tries on a fan this large): plain kernel with 32-thread blocks (table
    # and quad stencils), persistent kernel with 128-thread blocks
    ("c4", 1, 3, 1): {"bytes_per_launch": 21227520 + 1478144, "source_sha256": "2602d2aac951aea9"},
    ("c4", 1, 2, 1): {"bytes_per_launch": 4333312 + 483584, "source_sha256": "2602d2aac951aea9"},
    ("c4", 2, 3, 1): {"bytes_per_launch": 20590080 + 385792, "source_sha256": "2602d2aac951aea9"},
}
SMS = 152
FP32_LANES_PER_SM = 128
FP64_FMA_PER_SM_CLK = 2  # GB300: FP64 issue rate is 1/64 of FP32


def kernel_source_hash():
    """Hash of the kernel code (comments and whitespace removed, so that a
    comment edit does not invalidate a capture)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), encoding="utf-8") as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)  # block comments
        src = re.sub(r"//[^\n]*", " ", src)  # line comments (no URLs or // in strings here)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def captured_traffic(workload, cfg):
    """DRAM bytes per launch from the capture of this exact kernel, or None."""
    if cfg is None:
        return None
    rec = TRAFFIC.get((workload, int(cfg.kernel), int(cfg.stencil), int(cfg.lanes_per_ray)))
    if rec is None or rec["source_sha256"] != kernel_source_hash():
        return None
    return rec["bytes_per_launch"]


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    p.add_argument("--no-tune", action="store_true")
    p.add_argument("--kernel", choices=["plain", "persistent"], default=None,
                   help="fixed launch configuration instead of the autotuner")
    p.add_argument("--stencil", choices=["gather", "quad", "table"], default="quad")
    p.add_argument("--order", choices=["canonical", "elevation"], default="elevation")
    p.add_argument("--threads", type=int, default=128)
    p.add_argument("--blocks-per-sm", type=int, default=0,
                   help="persistent kernel with --kernel: resident blocks per SM (0 = occupancy limit)")
    p.add_argument("--lanes", type=int, default=0, choices=[0, 1, 2, 4],
                   help="lanes per ray with --kernel (0 = the library's choice)")
    p.add_argument("--workload", choices=["c2", "c4", "c4sub", "c5"], default="c2",
                   help="fan for the --profile and --one-ray modes: c2 = the anisotropic 24,840-ray fan "
                        "(the benchmark's workload), c4 = the 495,122-ray ionogram-synthesis batch, "
                        "c4sub = every eighth frequency of that batch (63,432 rays, for captures that "
                        "replay the kernel many times), c5 = small serving requests fused into one launch "
                        "(--profile only)")
    p.add_argument("--one-ray", type=int, default=None,
                   help="latency mode: trace only this canonical ray of the fan (alone) --steps times "
                        "and print its time per stage evaluation")
    p.add_argument("--profile", action="store_true",
                   help="warm-up launches then one launch, nothing else (for ncu captures)")
    p.add_argument("--profile-plan", choices=["none", "own-previous"], default="none",
                   help="with --profile: run the fan as a plan ordered longest-first by the costs of its "
                        "own previous execution (long factor 6, four-lane share on a second stream) "
                        "instead of one trace call")
    p.add_argument("--cpu-sample", type=int, default=0,
                   help="rays of the fan the CPU oracle baseline traces (0 = the whole fan)")
    p.add_argument("--serve-fuse", type=int, default=16384,
                   help="fuse_max_rays of the serving section's fused runs")
    p.add_argument("--serve-slots", type=int, default=8,
                   help="request server stream slots (requests in flight at once)")
    p.add_argument("--serve-seconds", type=float, default=4.0,
                   help="seconds of Poisson arrivals per offered load in the serving section (0 = skip)")
    p.add_argument("--no-batch", action="store_true",
                   help="skip the batched ionogram-synthesis section (495,122 rays in one captured graph)")
    p.add_argument("--rtol", type=float, default=1e-8,
                   help="RKF45 tolerance of the timed fan (the workload's 1e-8; a secondary "
                        "line is measured at ten times tighter)")
    return p.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id):
        self.rows, self.proc, self.th, self.device_id = [], None, None, device_id

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.device_id)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.th:
            self.th.join(timeout=5)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm, mx, reasons = [], None, set()
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def combine_ranks(mean_ms, n_rays, world):
    """Whole-job throughput of replicas: every rank traces its own fan of
    n_rays; the job takes as long as the slowest rank (max over ranks of the
    mean step time, reduced with the default process group when world > 1)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([mean_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        mean_ms = float(t.item())
    return mean_ms, n_rays * world / (mean_ms / 1e3)


def cpu_oracle_rate(workload, n_sample, seed=1234, single_core_rays=128):
    """The FP64 oracle as it stands on the host cores: all cores over a seeded
    sample of the fan (n_sample <= 0 or >= the fan: the whole fan, about 10 s
    on 16 Arm cores), and one core over the first rays of that sample."""
    from oracle import oracle
    oracle.build()
    g = oracle.Grid(workload.grid, workload.ne)
    n_all = workload.fan.n_rays
    if n_sample <= 0 or n_sample >= n_all:
        idx, what = np.arange(n_all), "the whole %d-ray fan" % n_all
    else:
        idx = np.sort(np.random.default_rng(seed).choice(n_all, n_sample, replace=False))
        what = "%d seeded rays of the %d-ray fan" % (n_sample, n_all)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    res = oracle.trace_fan(g, workload.fan, indices=idx, n_threads=cores)
    dt = time.perf_counter() - t0
    one = idx[:single_core_rays]
    t1 = time.perf_counter()
    res1 = oracle.trace_fan(g, workload.fan, indices=one, n_threads=1)
    dt1 = time.perf_counter() - t1
    info = dict(value=len(idx) / dt, unit="rays/s", cores=cores, kind="oracle",
                sample="%s (FP64 CPU oracle, %d threads)" % (what, cores),
                ray_steps_per_s=float(res["n_steps"].sum()) / dt, seconds=dt,
                single_core={"value": len(one) / dt1, "unit": "rays/s", "rays": len(one), "seconds": dt1,
                             "ray_steps_per_s": float(res1["n_steps"].sum()) / dt1})
    return info, idx, res


GATE_KM, GATE_DEG = 0.05, 1e-4
ERROR_FIELDS = ("group_path_km", "ground_range_km", "az_dev_deg", "apogee_km", "land_lat_deg", "land_lon_deg")


def gate_errors(r, ref, well, idx=None, km=GATE_KM, deg=GATE_DEG):
    """Per-output errors of records r (r[idx] when idx is given) against
    reference records ref: statuses over all rays; every output's max / p99 /
    p99.9 over the rays of `well` whose statuses agree; the share of those
    within the bar (P' and D within km; azimuth deviation within deg)."""
    g = r if idx is None else r[idx]
    mism = g["status"] != ref["status"]
    m = np.asarray(well, bool) & ~mism
    out = {"rays": int(len(ref)), "rays_compared": int(m.sum()), "status_mismatch": int(mism.sum())}
    if not m.any():
        return out
    inside = np.ones(int(m.sum()), bool)
    for f in ERROR_FIELDS:
        d = np.abs(g[f] - ref[f])[m]
        out[f] = {"max": float(d.max()), "p99": float(np.percentile(d, 99)), "p99.9": float(np.percentile(d, 99.9))}
        if f in ("group_path_km", "ground_range_km"):
            out[f]["within_bar"] = float(np.mean(d <= km))
            inside &= d <= km
        if f == "az_dev_deg":
            out[f]["within_bar"] = float(np.mean(d <= deg))
    out["bar"] = {"km": km, "deg": deg}
    out["p_and_d_within_bar_share"] = float(inside.mean())
    out["p_and_d_beyond_bar_rays"] = int((~inside).sum())
    return out


def oracle_well_conditioned(w, spec, o_idx, o_res):
    """Rays (of o_idx) not within 0.05 deg of a skip or Pedersen boundary, the
    boundaries located with the oracle alone; and a summary."""
    from oracle import boundaries as bd
    from oracle import oracle
    g = oracle.Grid(w.grid, w.ne)
    t0 = time.perf_counter()
    if len(o_idx) == spec.n_rays:
        near, n_b = bd.fan_exclusion(oracle, g, spec, o_res)
    else:
        near, n_b = bd.sample_exclusion(oracle, g, spec, o_idx, o_res)
    return ~near, {"located": int(n_b), "excluded_rays": int(near.sum()), "of_rays": int(len(near)),
                   "excluded_share": float(near.mean()), "seconds": time.perf_counter() - t0,
                   "rule": "within %.2f deg of elevation of a boundary located by oracle bisection to %.2f deg"
                           % (bd.EXCLUSION_DEG, bd.RESOLUTION_DEG)}


def tighter_rtol_gate(w, spec8, res8):
    """Records of the fan at the tighter rtol against the oracle's on every
    second azimuth, over the rays away from oracle-located boundaries."""
    from oracle import boundaries as bd
    from oracle import oracle
    g = oracle.Grid(w.grid, w.ne)
    n_a = len(spec8.az_deg)
    sub = spec8.replace(az_deg=spec8.az_deg[::2])
    idx = np.nonzero((np.arange(spec8.n_rays) % n_a) % 2 == 0)[0]
    t0 = time.perf_counter()
    ref = oracle.trace_fan(g, sub)
    near, n_b = bd.fan_exclusion(oracle, g, sub, ref)
    out = gate_errors(res8, ref, ~near, idx)
    out.update({"rtol": spec8.rtol, "rays_of_fan": int(len(idx)), "boundaries": int(n_b),
                "excluded_rays": int(near.sum()), "oracle_seconds": time.perf_counter() - t0})
    return out


def converged_sample(w, spec, res, o_idx, o_res, well, n_sample=1500, seed=77):
    """The integrator's own error: the mixed records and the oracle's records
    at the fan's rtol against the oracle at rtol 1e-11 (atol 1e-9 km) on a
    seeded sample of well-conditioned rays."""
    from oracle import oracle
    g = oracle.Grid(w.grid, w.ne)
    pos = np.nonzero(well)[0]
    pick = np.sort(np.random.default_rng(seed).choice(pos, min(n_sample, len(pos)), replace=False))
    rays = o_idx[pick]
    t0 = time.perf_counter()
    conv = oracle.trace_fan(g, spec.replace(rtol=1e-11, atol_km=1e-9), indices=rays)
    ok = np.ones(len(rays), bool)
    return {"rays": int(len(rays)), "reference": "oracle, rtol 1e-11, atol 1e-9 km",
            "this_path": gate_errors(res, conv, ok, rays), "oracle_same_rtol": gate_errors(o_res[pick], conv, ok),
            "seconds": time.perf_counter() - t0}


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    from paper_2506_18579_gb300 import workloads as wl
    from oracle import oracle
    oracle.build()
    w = wl.config2()
    g = oracle.Grid(w.grid, w.ne)
    cores = os.cpu_count() or 1
    per_step = max(cores * 4, 32)
    rng = np.random.default_rng(99)
    for _ in range(args.warmup):
        oracle.trace_fan(g, w.fan, indices=np.sort(rng.choice(w.fan.n_rays, cores, replace=False)),
                         n_threads=cores)
    times, steps = [], 0
    for _ in range(args.steps):
        idx = np.sort(rng.choice(w.fan.n_rays, per_step, replace=False))
        t0 = time.perf_counter()
        res = oracle.trace_fan(g, w.fan, indices=idx, n_threads=cores)
        times.append(time.perf_counter() - t0)
        steps += int(res["n_steps"].sum())
    total = sum(times)
    value = per_step * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": w.name, "rays": w.fan.n_rays, "precision": "fp64 (CPU oracle)",
                   "rtol": w.fan.rtol, "rays_per_step": per_step,
                   "l2": "not applicable (host cores)", "parallelism": "host threads"},
        "ray_steps_per_s": steps / total,
        "cpu_baseline": {"value": value, "unit": "rays/s", "cores": cores, "kind": "oracle",
                         "sample": "%d seeded rays per step of the %d-ray fan" % (per_step, w.fan.n_rays)},
        "e2e": {"value": value, "unit": "rays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2506_18579_gb300 import build as rtbuild
    from paper_2506_18579_gb300 import rtgd as rt
    from paper_2506_18579_gb300 import workloads as wl

    rtbuild.build()
    if args.workload == "c5":
        if not args.profile:
            raise SystemExit("--workload c5 is for the --profile mode (the serving section times it)")
        profile_fused(rt, wl, args.serve_fuse, max(args.warmup, 1) + 1)
        return
    if args.workload in ("c4", "c4sub") and not (args.profile or args.one_ray is not None):
        raise SystemExit("--workload c4 is for the --profile and --one-ray modes (the batch section times it)")
    w = wl.config2() if args.workload == "c2" else wl.config4()
    spec = w.fan.replace(rtol=args.rtol) if args.workload == "c2" else w.fan
    if args.workload == "c4sub":
        spec = spec.replace(freq_mhz=spec.freq_mhz[::8])
    prec = rt.RT_MIXED if args.precision == "mixed" else rt.RT_FP64
    grid = rt.Grid(w.grid, w.ne, table=(prec == rt.RT_MIXED and
                                        (args.kernel is None or args.stencil == "table")))
    fan = rt.Fan(spec, prec)
    n = fan.n_rays
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    out = torch.empty(n * 64, dtype=torch.uint8, device="cuda")
    cfg, tune_ms = None, None
    if args.kernel is not None:
        cfg = rt.launch_config(
            kernel=rt.RT_KERNEL_PLAIN if args.kernel == "plain" else rt.RT_KERNEL_PERSISTENT,
            stencil={"gather": rt.RT_STENCIL_GATHER, "quad": rt.RT_STENCIL_QUAD,
                     "table": rt.RT_STENCIL_TABLE}[args.stencil],
            block_threads=args.threads,
            order=rt.RT_ORDER_CANONICAL if args.order == "canonical" else rt.RT_ORDER_ELEVATION_FASTEST,
            blocks_per_sm=args.blocks_per_sm, lanes_per_ray=args.lanes)
    elif prec == rt.RT_MIXED and not args.no_tune:
        # timed on the whole fan: a strided sub-fan has other slowest rays
        cfg, tune_ms = rt.rt_tune(grid, fan, max_rays=n, stream=sptr)
    if args.one_ray is not None:
        run_one_ray(args, rt, wl, torch, grid, spec, prec, cfg)
        grid.close()
        return
    if args.profile:
        if args.profile_plan == "own-previous":
            plan = rt.Plan(grid, fan, cfg)
            plan.execute(out.data_ptr(), n, stream=sptr)
            n_long = plan.order(out.data_ptr(), spread=0, long_factor=6.0, stream=sptr)
            for _ in range(max(args.warmup, 1) + 1):
                plan.execute(out.data_ptr(), n, stream=sptr)
            torch.cuda.synchronize()
            plan.close()
            print(json.dumps({"profile_plan": "own-previous", "four_lane_rays": n_long}), flush=True)
        for _ in range(max(args.warmup, 1) + 1 if args.profile_plan == "none" else 0):
            rt.rt_trace_device(grid, fan, out.data_ptr(), n, cfg=cfg, stream=sptr)
        torch.cuda.synchronize()
        res = rt.results_view(out.cpu().numpy(), n)
        print(json.dumps({"profile_run": True, "rays": n, "evals": int(res["n_evals"].sum()),
                          "launches": max(args.warmup, 1) + 1}), flush=True)
        grid.close()
        return
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")  # > 129 MB L2

    def step():
        rt.rt_trace_device(grid, fan, out.data_ptr(), n, cfg=cfg, stream=sptr)

    peaks = rt.rt_measure_peaks()  # this GPU's FP32/FP64 FMA and L2 read ceilings (own kernels)
    args.warmup = max(args.warmup, 3)  # at least 3 untimed warm-up steps
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    try:
        dev_id = torch.cuda.get_device_properties(local_rank).uuid
        dev_id = "GPU-" + str(dev_id) if not str(dev_id).startswith("GPU-") else str(dev_id)
    except Exception:
        dev_id = local_rank
    clocks = ClockSampler(dev_id)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()  # evict the grid and tables from L2 between timed steps
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    ms = [a.elapsed_time(b) for a, b in ev]
    mean_ms, job_rays_per_s = combine_ranks(float(np.mean(ms)), n, world)
    res = rt.results_view(out.cpu().numpy(), n)
    ray_steps = int(res["n_steps"].sum())
    attempts = int(res["n_attempts"].sum())
    evals = int(res["n_evals"].sum())

    # end to end through the public call: fan arrays from the host, results
    # into pinned host memory, synchronised, every step
    pinned = torch.empty(n * 64, dtype=torch.uint8, pin_memory=True)
    host_out = pinned.numpy().view(rt.RESULT_DTYPE)
    e2e_t = []
    for i in range(max(3, min(args.steps, 10))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rt.rt_trace(grid, fan, out=host_out, cfg=cfg, stream=sptr)
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = float(np.mean(e2e_t[1:]))

    line = None
    if rank == 0:
        # the FP64 path's own throughput at this tolerance, and its records
        t0 = time.perf_counter()
        ref64 = rt.rt_trace(grid, rt.Fan(spec, rt.RT_FP64), stream=sptr)
        fp64_s = time.perf_counter() - t0
        conv = rt.rt_trace(grid, rt.Fan(w.fan.replace(rtol=1e-11, atol_km=1e-9), rt.RT_FP64), stream=sptr)
        # ten times tighter tolerance: throughput of the same path
        spec8 = spec.replace(rtol=args.rtol / 10.0)
        fan8 = rt.Fan(spec8, prec)
        out8 = torch.empty(n * 64, dtype=torch.uint8, device="cuda")
        cfg8 = cfg
        if args.kernel is None and prec == rt.RT_MIXED and not args.no_tune:
            cfg8, _ = rt.rt_tune(grid, fan8, max_rays=n, stream=sptr)
        for _ in range(2):
            rt.rt_trace_device(grid, fan8, out8.data_ptr(), n, cfg=cfg8, stream=sptr)
        t8 = []
        for _ in range(5):
            flush.zero_()
            a8, b8 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a8.record(stream)
            rt.rt_trace_device(grid, fan8, out8.data_ptr(), n, cfg=cfg8, stream=sptr)
            b8.record(stream)
            torch.cuda.synchronize()
            t8.append(a8.elapsed_time(b8))
        res8 = rt.results_view(out8.cpu().numpy(), n).copy()
        nominal = {"rtol": args.rtol / 10.0, "rays_per_s": n / (np.mean(t8) / 1e3), "ms_per_step": float(np.mean(t8)),
                   "ray_steps_per_s": float(res8["n_steps"].sum()) / (np.mean(t8) / 1e3)}
        richardson = (richardson_table(rt, wl, grid, spec, prec, cfg, sptr) if args.workload == "c2" else None)
        cpu, acc = None, {"vs_richardson": richardson}
        if world == 1:
            # the CPU baseline leg traces the fan through the oracle; its records
            # give the full-size parity of both GPU paths, and the oracle alone
            # locates the skip / Pedersen boundaries that the mixed bar excludes
            cpu, o_idx, o_res = cpu_oracle_rate(w, args.cpu_sample)
            well, gate_info = oracle_well_conditioned(w, spec, o_idx, o_res)
            acc["boundaries"] = gate_info
            acc["vs_cpu_oracle"] = gate_errors(res, o_res, well, o_idx)
            acc["fp64_gpu_vs_cpu_oracle"] = gate_errors(ref64, o_res, np.ones(len(o_idx), bool), o_idx,
                                                         km=1e-6, deg=1e-7)
            # the same fan at ten times tighter rtol against the oracle there
            # (every second azimuth)
            acc["tighter_rtol_vs_cpu_oracle"] = tighter_rtol_gate(w, spec8, res8)
            # how far both paths are from a converged oracle run (rtol 1e-11) on a
            # seeded sample of well-conditioned rays: the integrator's own error
            acc["vs_converged_oracle"] = converged_sample(w, spec, res, o_idx, o_res, well)
        # against the GPU FP64 path (the comparison baseline) over the same rays
        well_all = np.ones(n, bool)
        if world == 1 and len(o_idx) == n:
            well_all = well
        acc["vs_fp64_same_rtol"] = gate_errors(res, ref64, well_all)
        acc["fp64_same_rtol_vs_converged_fp64_gpu"] = gate_errors(ref64, conv, well_all)
        acc["vs_converged_fp64_gpu"] = gate_errors(res, conv, well_all)
        acc["well_conditioned"] = ("rays not within 0.05 deg of elevation of a skip or Pedersen boundary "
                                   "located with the oracle" if world == 1 else "all rays (no CPU leg at N > 1)")
        sec = mean_ms / 1e3
        flop = evals * FLOP_PER_EVAL[args.precision]
        if prec == rt.RT_MIXED:
            peak = SMS * FP32_LANES_PER_SM * 2 * 2070e6 / 1e12
            bound_note = "FP32 issue: 152 SMs x 128 lanes x 2 flop x 2070 MHz"
        else:
            peak = SMS * FP64_FMA_PER_SM_CLK * 2 * 2070e6 / 1e12
            bound_note = "FP64: 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz"
        achieved = flop / sec / 1e12
        # the fan's critical path: its longest ray traced alone, same launch configuration
        i_long = int(np.argmax(res["n_evals"]))
        alone_ms, _ = time_one_ray(rt, torch, grid, one_ray_spec(wl, spec, i_long), prec, cfg, 3, 2)
        critical = {"longest_ray_alone_ms": alone_ms, "fan_ms": mean_ms, "fan_over_alone": mean_ms / alone_ms,
                    "ns_per_stage_eval_alone": alone_ms * 1e6 / max(int(res["n_evals"][i_long]), 1)}
        # the FP64 path's own critical path: its longest ray traced alone (one
        # thread per ray), beside its whole-fan time
        fp64_alone = None
        if prec == rt.RT_MIXED:
            i64 = int(np.argmax(ref64["n_evals"]))
            a64, r64 = time_one_ray(rt, torch, grid, one_ray_spec(wl, spec, i64), rt.RT_FP64, None, 1, 1)
            fp64_alone = {"longest_ray_alone_ms": a64, "stage_evals": int(r64["n_evals"][0]),
                          "ns_per_stage_eval_alone": a64 * 1e6 / max(int(r64["n_evals"][0]), 1),
                          "fan_over_alone": fp64_s * 1e3 / a64}
        # the same fan as a plan ordered by earlier costs (a repeated scan)
        fan_ordered = None
        if prec == rt.RT_MIXED and cfg is not None and args.workload == "c2":
            try:
                fan_ordered = run_fan_ordered(rt, wl, torch, grid, fan, spec, cfg, flush, res,
                                              o_res if world == 1 and len(o_idx) == n else None,
                                              well_all if world == 1 and len(o_idx) == n else None)
            except Exception as exc:
                fan_ordered = {"error": repr(exc)}
        batch = None
        if world == 1 and not args.no_batch and prec == rt.RT_MIXED:
            try:
                batch = run_batch(rt, wl, torch, flush)
            except Exception as exc:
                batch = {"error": repr(exc)}
        interpolants = None
        if world == 1 and not args.no_batch:
            try:
                interpolants = run_interpolants(rt, wl)
            except Exception as exc:
                interpolants = {"error": repr(exc)}
        serving = None
        if world == 1 and args.serve_seconds > 0 and prec == rt.RT_MIXED:
            try:
                serving = run_serving(rt, wl, args.serve_seconds, slots=args.serve_slots, fuse=args.serve_fuse)
            except Exception as exc:  # the serving section must not cost the main line
                serving = {"error": repr(exc)}
        line = {
            "metric": METRIC, "value": job_rays_per_s, "unit": "rays/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if prec == rt.RT_MIXED else "f64", "data": "synthetic",
            "config": {"workload": w.name, "rays": n, "precision": args.precision, "rtol": args.rtol,
                       "launch": None if cfg is None else {"kernel": cfg.kernel, "stencil": cfg.stencil,
                                                           "block_threads": cfg.block_threads,
                                                           "order": cfg.order,
                                                           "lanes_per_ray": cfg.lanes_per_ray},
                       "l2": "flushed (512 MiB write) before every timed step",
                       "parallelism": "replicas" if world > 1 else "single"},
            "ray_steps_per_s": ray_steps * world / sec,
            "attempts_per_s": attempts * world / sec,
            "stage_evals_per_s": evals * world / sec,
            "fan_latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99))},
            "critical_path": critical,
            "fan_ordered": fan_ordered,
            "longest_ray": {"index": int(np.argmax(res["n_evals"])), "stage_evals": int(res["n_evals"].max()),
                            "status": int(res["status"][int(np.argmax(res["n_evals"]))]),
                            "stage_evals_p50": float(np.median(res["n_evals"])),
                            "stage_evals_p99": float(np.percentile(res["n_evals"], 99))},
            "accuracy": acc,
            "tighter_rtol": nominal,
            "fp64_gpu_path": {"rays_per_s": n / fp64_s, "seconds": fp64_s, "critical_path": fp64_alone},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": captured_traffic(args.workload, cfg),
                         "traffic_unit": "bytes per launch (DRAM read + write, ncu)",
                         "kernel_source_sha256": kernel_source_hash(), "peak_basis": bound_note,
                         "flop_per_stage_eval": FLOP_PER_EVAL[args.precision],
                         "measured_peaks": peaks,
                         "frac_of_measured": achieved / (peaks["fp32_fma_tflops"] if prec == rt.RT_MIXED
                                                         else peaks["fp64_fma_tflops"]),
                         "gather": {"bytes_per_stage_eval": GATHER_BYTES[args.precision],
                                    "achieved_gbs": evals * GATHER_BYTES[args.precision] / sec / 1e9,
                                    "l2_read_peak_gbs": peaks["l2_read_gbs"]},
                         # the fan leaves most of the GPU idle: its floor is its longest
                         # ray's dependent chain of stage evaluations, traced alone
                         "latency_floor": {"longest_ray_alone_ms": alone_ms, "fan_ms": mean_ms,
                                           "frac": alone_ms / mean_ms}},
            "cpu_baseline": cpu,
            "e2e": {"value": n * world / e2e_s, "unit": "rays/s", "h2d_bytes_per_step": fan.host_bytes,
                    "d2h_bytes_per_step": n * 64},
            "gpu_launches": args.steps * (2 if prec == rt.RT_MIXED else 1),  # trace (+ finish pass) per step
            "clocks": clk,
            "wall_s_timed": t_wall,
            "tune_ms": tune_ms,
            "batch": batch,
            "interpolants": interpolants,
            "serving": serving,
        }
    grid.close()
    if line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def one_ray_spec(wl, spec, index):
    """The fan of spec reduced to its canonical ray `index` (a one-ray fan)."""
    freq, el, az = np.atleast_1d(spec.freq_mhz), np.atleast_1d(spec.el_deg), np.atleast_1d(spec.az_deg)
    modes = [m for m in (wl.MODE_O, wl.MODE_X) if spec.modes & m]
    i = index
    ia, i = i % len(az), i // len(az)
    ie, i = i % len(el), i // len(el)
    im, fi = i % len(modes), i // len(modes)
    return spec.replace(freq_mhz=np.array([freq[fi]]), modes=modes[im], el_deg=np.array([el[ie]]),
                        az_deg=np.array([az[ia]]))


def richardson_extrapolate(y_h, y_h2, y_h4, floor=1e-9):
    """Richardson extrapolation of three runs at steps h, h/2, h/4: the
    observed order p = median over entries of log2(|y_h - y_h2| / |y_h2 -
    y_h4|) (entries whose last difference is below `floor` are rounding and
    left out; p = 4 if none remain), and the extrapolated values y_h4 +
    (y_h4 - y_h2) / (2^p - 1).  Returns (extrapolated, p)."""
    y_h, y_h2, y_h4 = (np.asarray(a, dtype=np.float64) for a in (y_h, y_h2, y_h4))
    d1, d2 = np.abs(y_h - y_h2), np.abs(y_h2 - y_h4)
    big = d2 > floor
    p = float(np.median(np.log2(d1[big] / d2[big]))) if big.any() else 4.0
    return y_h4 + (y_h4 - y_h2) / (2.0 ** p - 1.0), p


def richardson_table(rt, wl, grid, spec, prec, cfg, stream):
    """Per-output errors against a Richardson-extrapolated reference (Sec.
    IV-B) on a regular sub-fan of the fan (every 5th elevation, every 4th
    azimuth: 1,242 rays of C2).  Reference: fixed-step RK4 in FP64 at h = 1,
    0.5 and 0.25 km, extrapolated as y(h/4) + (y(h/4) - y(h/2)) / (2^p - 1)
    with p the observed order, median of log2(|y(h) - y(h/2)| / |y(h/2) -
    y(h/4)|) over the rays.  p comes out near 2, not 4: the GD field's
    gradient is only continuous across cell faces, and a fixed step that
    straddles a face loses the fourth-order local error (the adaptive path
    ends its steps at faces).  Rays that land or escape (their end point is
    solved, not cut at a step) with the same status in every run are
    compared."""
    sub = spec.replace(el_deg=np.asarray(spec.el_deg)[::5], az_deg=np.asarray(spec.az_deg)[::4])
    runs = [rt.rt_trace(grid, rt.Fan(sub.replace(integrator=wl.RK4, h_km=h, max_steps=400000), rt.RT_FP64),
                        stream=stream) for h in (1.0, 0.5, 0.25)]
    ours = rt.rt_trace(grid, rt.Fan(sub, prec), cfg=cfg, stream=stream)
    same_rtol = rt.rt_trace(grid, rt.Fan(sub, rt.RT_FP64), stream=stream)
    conv = rt.rt_trace(grid, rt.Fan(sub.replace(rtol=1e-11, atol_km=1e-9), rt.RT_FP64), stream=stream)
    st = runs[2]["status"]
    ok = np.isin(st, (rt.RT_RAY_LANDED, rt.RT_RAY_ESCAPED))
    for r in runs[:2] + [ours, same_rtol, conv]:
        ok &= r["status"] == st
    fields = ("group_path_km", "ground_range_km", "az_dev_deg", "apogee_km")
    _, order = richardson_extrapolate(*(r["group_path_km"][ok] for r in runs))
    ref = {f: runs[2][f] + (runs[2][f] - runs[1][f]) / (2.0 ** order - 1.0) for f in fields}

    def err(r):
        return {f: {"max": float(np.abs(r[f] - ref[f])[ok].max()),
                    "p99": float(np.percentile(np.abs(r[f] - ref[f])[ok], 99))} for f in fields}

    return {"rays": int(sub.n_rays), "rays_compared": int(ok.sum()),
            "reference": "RK4 FP64, h = 1 / 0.5 / 0.25 km, Richardson-extrapolated at the observed order",
            "observed_order_group_path": order,
            "this_path": err(ours), "fp64_same_rtol": err(same_rtol), "fp64_rtol_1e-11": err(conv),
            "rk4_h_0.25_km": err(runs[2])}


def run_fan_ordered(rt, wl, torch, grid, fan, spec, cfg, flush, res, o_res, well, steps=7,
                    long_factor=2.0):
    """The fan as a plan whose rays are ordered by the costs of an earlier
    trace (rt_plan_order): the rays above long_factor x the median cost at
    four lanes, a warp each, on SMs of their own (RT_PLAN_LONG_EXCLUSIVE |
    RT_PLAN_LONG_ALONE), the rest in the plan's own order.  Cost sources: the
    plan's previous execution (a scan repeated on the same ionosphere) and the
    same scan on a later snapshot (the TID advanced 5 % of its period).
    Every execution traces every ray; records are compared with the
    canonical fan's and, where given, with the oracle's."""
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    n = fan.n_rays
    plan = rt.Plan(grid, fan, cfg)
    own = torch.empty(n * 64, dtype=torch.uint8, device="cuda")
    plan.execute(own.data_ptr(), n, stream=sptr)
    w_snap = wl.config2(tid_phase_shift=0.05)
    g_snap = rt.Grid(w_snap.grid, w_snap.ne, table=True)
    snap = torch.empty(n * 64, dtype=torch.uint8, device="cuda")
    rt.rt_trace_device(g_snap, rt.Fan(spec, rt.RT_MIXED), snap.data_ptr(), n, cfg=cfg, stream=sptr)
    torch.cuda.synchronize()
    g_snap.close()
    out = torch.empty(n * 64, dtype=torch.uint8, device="cuda")
    ref_bytes = np.ascontiguousarray(res).tobytes()
    result = {"long_factor": long_factor, "flags": "RT_PLAN_LONG_EXCLUSIVE | RT_PLAN_LONG_ALONE | "
                                                   "RT_PLAN_REST_IN_PLAN_ORDER",
              "l2": "flushed before every execution"}
    for name, src, spread in (("own_previous", own, 0), ("later_snapshot", snap, 1)):
        n_long = plan.order(src.data_ptr(), spread=spread, long_factor=long_factor, rest_in_plan_order=True,
                            long_exclusive=True, long_alone=True, stream=sptr)
        for _ in range(2):
            plan.execute(out.data_ptr(), n, stream=sptr)
        ms = []
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            plan.execute(out.data_ptr(), n, stream=sptr)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        rec = rt.results_view(out.cpu().numpy(), n).copy()
        entry = {"ms_per_fan": float(np.mean(ms)), "rays_per_s": n / (float(np.mean(ms)) / 1e3),
                 "fan_latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99))},
                 "four_lane_rays": int(n_long), "spread": spread,
                 "records_identical_to_the_canonical_fan": rec.tobytes() == ref_bytes}
        if o_res is not None:
            entry["vs_cpu_oracle"] = gate_errors(rec, o_res, well)
        result[name] = entry
    result["cost_sources"] = {"own_previous": "the plan's previous execution (same ionosphere)",
                              "later_snapshot": "the same scan on the ionosphere with the TID advanced by 5 % "
                                                "of its period"}
    plan.close()
    return result


def time_one_ray(rt, torch, grid, one, prec, cfg, steps, warmup):
    """Median CUDA-event time (ms) of tracing a one-ray fan alone, and its record."""
    fan = rt.Fan(one, prec)
    st = torch.cuda.current_stream()
    buf = torch.empty(64, dtype=torch.uint8, device="cuda")
    for _ in range(max(warmup, 1)):
        rt.rt_trace_device(grid, fan, buf.data_ptr(), 1, cfg=cfg, stream=st.cuda_stream)
    ts = []
    for _ in range(steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        rt.rt_trace_device(grid, fan, buf.data_ptr(), 1, cfg=cfg, stream=st.cuda_stream)
        b.record(st)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts)), rt.results_view(buf.cpu().numpy(), 1).copy()


def run_one_ray(args, rt, wl, torch, grid, spec, prec, cfg):
    """Latency of one ray traced alone (a one-ray fan): the fan's critical path
    when its longest ray dominates.  Prints the time per stage evaluation."""
    one = one_ray_spec(wl, spec, args.one_ray)
    ms, r = time_one_ray(rt, torch, grid, one, prec, cfg, args.steps, args.warmup)
    print(json.dumps({"one_ray": args.one_ray, "freq_mhz": float(one.freq_mhz[0]),
                      "mode": "O" if one.modes == wl.MODE_O else "X",
                      "el_deg": float(one.el_deg[0]), "az_deg": float(one.az_deg[0]), "status": int(r["status"][0]),
                      "stage_evals": int(r["n_evals"][0]), "ms": ms,
                      "ns_per_stage_eval": ms * 1e6 / max(int(r["n_evals"][0]), 1),
                      "launch": None if cfg is None else {"kernel": cfg.kernel, "stencil": cfg.stencil,
                                                          "lanes_per_ray": cfg.lanes_per_ray}}), flush=True)


def run_batch(rt, wl, torch, flush, steps=3):
    """Batched form: the ionogram-synthesis batch (181x361x301 grid, 281
    frequencies x 881 elevations x O/X = 495,122 rays of 50-5000 steps) as one
    autotuned plan captured in a CUDA graph; L2 flushed before each replay."""
    w = wl.config4()
    grid = rt.Grid(w.grid, w.ne, table=True)  # 5 GB per-cell table: a tuner candidate
    fan = rt.Fan(w.fan, rt.RT_MIXED)
    n = fan.n_rays
    side = torch.cuda.Stream()
    cfg, tune_ms = rt.rt_tune(grid, fan, max_rays=65536, stream=side.cuda_stream)
    plan = rt.Plan(grid, fan, cfg=cfg)
    out = torch.empty(n * 64, dtype=torch.uint8, device="cuda")
    graph = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            plan.execute(out.data_ptr(), n, stream=side.cuda_stream)
    torch.cuda.synchronize()
    cur = torch.cuda.current_stream()
    graph.replay()
    torch.cuda.synchronize()
    ms = []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(cur)
        graph.replay()
        b.record(cur)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    res = rt.results_view(out.cpu().numpy(), n)
    out_first = out.clone()
    st = np.bincount(res["status"], minlength=8)
    sec = float(np.mean(ms)) / 1e3
    out_d = {"workload": w.name, "rays": n, "rtol": w.fan.rtol, "ms_per_batch": sec * 1e3, "rays_per_s": n / sec,
             "ray_steps_per_s": float(res["n_steps"].sum()) / sec,
             "stage_evals_per_s": float(res["n_evals"].sum()) / sec,
             "steps_per_ray": {"min": int(res["n_steps"].min()), "p50": float(np.median(res["n_steps"])),
                               "max": int(res["n_steps"].max())},
             "status_counts": {"landed": int(st[rt.RT_RAY_LANDED]), "escaped": int(st[rt.RT_RAY_ESCAPED]),
                               "left_grid": int(st[rt.RT_RAY_LEFT_GRID]), "other": int(n - st[1:4].sum())},
             "launch": {"kernel": cfg.kernel, "stencil": cfg.stencil, "block_threads": cfg.block_threads,
                        "order": cfg.order, "lanes_per_ray": cfg.lanes_per_ray},
             "graph": "one plan execute (counter reset + launch) captured, replayed per batch",
             "tune_ms": tune_ms, "l2": "flushed before every replay",
             "cpu_baseline": None, "vs_cpu_oracle": None,
             "roofline": {"bound": "alu", "achieved": float(res["n_evals"].sum()) * FLOP_PER_EVAL["mixed"] / sec / 1e12,
                          "peak": SMS * FP32_LANES_PER_SM * 2 * 2070e6 / 1e12, "unit": "TFLOP/s",
                          "traffic": captured_traffic("c4", cfg)}}
    out_d["roofline"]["frac"] = out_d["roofline"]["achieved"] / out_d["roofline"]["peak"]
    # oblique-ionogram synthesis on the batch's grid and scan (Sec. IV-B-4):
    # transmitter to a receiver 1,500 km away along azimuth 45 deg; one blocking
    # rt_ionogram call (trace, point extraction on the GPU, host sort)
    lat1, lon1, brg, dd = np.radians(w.fan.tx_lat_deg), np.radians(w.fan.tx_lon_deg), np.radians(45.0), 1500.0 / 6371.0
    lat2 = np.arcsin(np.sin(lat1) * np.cos(dd) + np.cos(lat1) * np.sin(dd) * np.cos(brg))
    lon2 = lon1 + np.arctan2(np.sin(brg) * np.sin(dd) * np.cos(lat1), np.cos(dd) - np.sin(lat1) * np.sin(lat2))
    rx = (float(np.degrees(lat2)), float(np.degrees(lon2)))
    iono_kw = dict(modes=w.fan.modes, integrator=w.fan.integrator, precision=rt.RT_MIXED, rtol=w.fan.rtol,
                   atol_km=w.fan.atol_km, h_km=w.fan.h_km, h_max_km=w.fan.h_max_km, cfg=cfg)
    tx = (w.fan.tx_lat_deg, w.fan.tx_lon_deg, w.fan.tx_alt_km)
    rt.rt_ionogram(grid, tx, rx, w.fan.freq_mhz, w.fan.el_deg, **iono_kw)  # warm-up
    t_io = []
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pts, n_pts = rt.rt_ionogram(grid, tx, rx, w.fan.freq_mhz, w.fan.el_deg, **iono_kw)
        t_io.append(time.perf_counter() - t0)
    out_d["ionogram"] = {"receiver_km": 1500.0, "rays": n, "points": int(n_pts),
                         "ms_per_ionogram": float(np.mean(t_io)) * 1e3,
                         "traces_with_points": int(len({(float(p["freq_mhz"]), int(p["mode"])) for p in pts}))}
    # the same batch as one persistent launch (lane groups claim rays from an
    # atomic counter), captured and replayed like the tuned plan
    cfg_p = rt.launch_config(kernel=rt.RT_KERNEL_PERSISTENT, stencil=cfg.stencil, block_threads=cfg.block_threads,
                             order=cfg.order, lanes_per_ray=cfg.lanes_per_ray)
    pplan = rt.Plan(grid, fan, cfg=cfg_p)
    pgraph = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        with torch.cuda.graph(pgraph, stream=side):
            pplan.execute(out.data_ptr(), n, stream=side.cuda_stream)
    torch.cuda.synchronize()
    pgraph.replay()
    t_p = []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(cur)
        pgraph.replay()
        b.record(cur)
        torch.cuda.synchronize()
        t_p.append(a.elapsed_time(b))
    out_d["persistent_graph"] = {"ms_per_batch": float(np.mean(t_p)), "rays_per_s": n / (float(np.mean(t_p)) / 1e3),
                                 "launch": {"kernel": cfg_p.kernel, "stencil": cfg_p.stencil,
                                            "block_threads": cfg_p.block_threads, "order": cfg_p.order,
                                            "lanes_per_ray": cfg_p.lanes_per_ray}}
    del pgraph
    pplan.close()
    # longest-first (rt_plan_order): the costs come from the same scan traced
    # on a later snapshot of the ionosphere (the TID advanced by 5 % of its
    # period, about a minute for a 200 km TID at 150 m/s), as a scan repeated on
    # successive snapshots has them, or from the plan's own previous execution
    # (the same ionosphere); the most expensive rays (six times the median
    # cost) run at four lanes each on a second stream, all in descending cost
    w5 = wl.config4(tid_phase_shift=0.05)
    g5 = rt.Grid(w5.grid, w5.ne)
    prev = torch.empty(n * 64, dtype=torch.uint8, device="cuda")
    rt.rt_trace_device(g5, rt.Fan(w5.fan, rt.RT_MIXED), prev.data_ptr(), n,
                       cfg=rt.launch_config(kernel=rt.RT_KERNEL_PLAIN, stencil=rt.RT_STENCIL_QUAD, lanes_per_ray=1),
                       stream=side.cuda_stream)
    own = torch.empty(n * 64, dtype=torch.uint8, device="cuda")
    own.copy_(out_first)
    torch.cuda.synchronize()
    g5.close()
    out_d["ordered"] = {"spread": {"later_snapshot": 1, "own_previous": 0}, "long_factor": 6.0,
                        "flags": "RT_PLAN_LONG_EXCLUSIVE (the four-lane share on SMs of its own)",
                        "cost_sources": {"later_snapshot": "the same scan on the ionosphere with the TID advanced by "
                                                           "5 % of its period",
                                         "own_previous": "the plan's previous execution (same ionosphere)"}}
    ordered_sample = {}
    # spread: the costs of a later snapshot are dilated over one elevation and
    # frequency step (boundaries move); the plan's own previous costs are exact
    for name, c, src, spread in (("plain", cfg, prev, 1), ("persistent", cfg_p, prev, 1),
                                 ("plain_own_previous", cfg, own, 0), ("persistent_own_previous", cfg_p, own, 0)):
        oplan = rt.Plan(grid, fan, cfg=c)
        n_long = oplan.order(src.data_ptr(), spread=spread, long_factor=6.0, long_exclusive=True,
                             stream=side.cuda_stream)
        ograph = torch.cuda.CUDAGraph()
        torch.cuda.synchronize()
        with torch.cuda.stream(side):
            with torch.cuda.graph(ograph, stream=side):
                oplan.execute(out.data_ptr(), n, stream=side.cuda_stream)
        torch.cuda.synchronize()
        ograph.replay()
        t_o = []
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(cur)
            ograph.replay()
            b.record(cur)
            torch.cuda.synchronize()
            t_o.append(a.elapsed_time(b))
        res_o = rt.results_view(out.cpu().numpy(), n)
        ordered_sample[name] = res_o[wl.sample_indices(n, 5000, 1234)].copy()  # the oracle leg's sample
        out_d["ordered"][name] = {"ms_per_batch": float(np.mean(t_o)), "rays_per_s": n / (float(np.mean(t_o)) / 1e3),
                                  "four_lane_rays": int(n_long), "spread": spread,
                                  "stage_evals_per_s": float(res_o["n_evals"].sum()) / (float(np.mean(t_o)) / 1e3),
                                  "launch": {"kernel": c.kernel, "stencil": c.stencil, "block_threads": c.block_threads,
                                             "lanes_per_ray": c.lanes_per_ray}}
        del ograph
        oplan.close()
    del prev, own
    # cost of the interpolant (Sec. IV: GD against Catmull-Rom): the same batch,
    # the same launch configuration, on a Catmull-Rom copy of the grid; time
    # per stage evaluation (the two fields differ slightly, so do the paths)
    grid_cr = rt.Grid(w.grid, w.ne, interp="cr", table=(cfg.stencil == rt.RT_STENCIL_TABLE))
    t_cr = []
    for i in range(steps + 1):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(cur)
        rt.rt_trace_device(grid_cr, fan, out.data_ptr(), n, cfg=cfg, stream=cur.cuda_stream)
        b.record(cur)
        torch.cuda.synchronize()
        if i > 0:
            t_cr.append(a.elapsed_time(b))
    res_cr = rt.results_view(out.cpu().numpy(), n)
    ns_gd = sec * 1e9 / float(res["n_evals"].sum())
    ns_cr = float(np.mean(t_cr)) * 1e6 / float(res_cr["n_evals"].sum())
    out_d["interpolant_cost"] = {"gd_ns_per_stage_eval": ns_gd, "cr_ns_per_stage_eval": ns_cr,
                                 "gd_over_cr": ns_gd / ns_cr, "cr_ms_per_batch": float(np.mean(t_cr))}
    grid_cr.close()
    # CPU baseline leg of the batch: the FP64 oracle on a seeded 5,000-ray
    # sample (its rays/s stands for the whole batch), and the batch's mixed
    # records against the oracle's on that sample, over the sampled rays not
    # within 0.05 deg of a boundary the oracle locates around them
    info, idx, o_res = cpu_oracle_rate(w, 5000)
    well, gate_info = oracle_well_conditioned(w, w.fan, idx, o_res)
    out_d["cpu_baseline"] = info
    out_d["boundaries"] = gate_info
    out_d["vs_cpu_oracle"] = gate_errors(res, o_res, well, idx)
    for name, rec in ordered_sample.items():
        out_d["ordered"][name]["vs_cpu_oracle"] = gate_errors(rec, o_res, well)
    del graph
    plan.close()
    grid.close()
    return out_d


def run_interpolants(rt, wl):
    """Accuracy of GD against Catmull-Rom (Sec. IV): one analytic ionosphere
    sampled on a coarse grid (1 deg, 1 deg, 5 km) and on a 4x finer grid that
    stands in for the analytic field; 3,232 rays traced on the FP64 path at
    rtol 1e-9 on the coarse grid with each interpolant, against the oracle
    with GD on the fine grid (the reference).  Errors over rays with the
    reference's status on both and not within 0.05 deg of a boundary the
    oracle locates on the fine grid."""
    from oracle import boundaries as bd
    from oracle import oracle
    c, nc, f, nf, spec = wl.interp_comparison()
    fan = rt.Fan(spec, rt.RT_FP64)
    grids = {"gd": rt.Grid(c, nc.astype(np.float64)), "cr": rt.Grid(c, nc.astype(np.float64), interp="cr")}
    res = {k: rt.rt_trace(gr, fan) for k, gr in grids.items()}
    og = oracle.Grid(f, nf)
    ref = oracle.trace_fan(og, spec)
    near, _ = bd.fan_exclusion(oracle, og, spec, ref)
    ok = ~near & (res["gd"]["status"] == ref["status"]) & (res["cr"]["status"] == ref["status"])
    out = {"grids": {"coarse": list(c.shape), "reference": list(f.shape)}, "rays": spec.n_rays,
           "reference": "oracle, GD on the 4x finer grid", "rays_compared": int(ok.sum())}
    for k in ("gd", "cr"):
        e = {}
        for fld in ("group_path_km", "ground_range_km", "apogee_km"):
            d = np.abs(res[k][fld] - ref[fld])[ok]
            e[fld] = {"max": float(d.max()), "median": float(np.median(d)), "rms": float(np.sqrt(np.mean(d ** 2)))}
        e["status_differs"] = int((res[k]["status"] != ref["status"]).sum())
        out[k] = e
    for gr in grids.values():
        gr.close()
    return out


def small_fans_compare(rt, wl, reps=5):
    """The same 64 small fans (1-2,000 rays each, from the serving mix on the
    91x181x151 grid) traced three ways: one launch per fan on one stream, one
    launch per fan spread over 8 streams, and one rt_trace_fans_device
    launch.  Median wall time of `reps` rounds, CUDA events around each
    round; rays/s of each way."""
    import torch

    grids = wl.serving_grids()
    gi = 2
    spec_g, ne = grids[gi]
    h = rt.Grid(spec_g, ne)
    small = [f for g, f in wl.serving_requests(2000, 9, [g for g, _ in grids])
             if g == gi and rt.Fan(f).n_rays <= 2000][:64]
    fans = [rt.Fan(f) for f in small]
    sizes = [f.n_rays for f in fans]
    n = sum(sizes)
    off = np.concatenate([[0], np.cumsum(sizes)])
    out = torch.empty(n * 64, dtype=torch.uint8, device="cuda")
    main = torch.cuda.current_stream()
    side = [torch.cuda.Stream() for _ in range(8)]
    cfg4 = rt.launch_config(kernel=rt.RT_KERNEL_PLAIN, stencil=rt.RT_STENCIL_QUAD, lanes_per_ray=4)

    def per_fan(streams):
        for k, f in enumerate(fans):
            st = streams[k % len(streams)]
            rt.rt_trace_device(h, f, out.data_ptr() + int(off[k]) * 64, sizes[k], cfg=cfg4, stream=st.cuda_stream)

    def fused(_):
        rt.rt_trace_fans_device(h, fans, out.data_ptr(), n, cfg=rt.launch_config(stencil=rt.RT_STENCIL_QUAD),
                                stream=main.cuda_stream)

    res = {}
    for name, fn, streams in (("one_launch_per_fan_1_stream", per_fan, [main]),
                              ("one_launch_per_fan_8_streams", per_fan, side),
                              ("one_fused_launch", fused, None)):
        ts = []
        for rep in range(reps + 1):
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(main)
            if streams is side:
                for st in side:
                    st.wait_event(a)
            fn(streams)
            if streams is side:
                for st in side:
                    main.wait_stream(st)
            b.record(main)
            torch.cuda.synchronize()
            if rep > 0:  # the first round warms up
                ts.append(a.elapsed_time(b))
        ms = float(np.median(ts))
        res[name] = {"ms": ms, "rays_per_s": n / (ms / 1e3)}
    h.close()
    return {"fans": len(fans), "rays": int(n), "grid": list(spec_g.shape), **res}


def profile_fused(rt, wl, fuse, rounds):
    """For ncu: `rounds` rounds on the 91x181x151 serving grid, each one large
    request (which runs unfused and keeps the one slot busy) followed by 64
    small requests, which queue behind it and go out as fused launches of at
    most `fuse` rays."""
    grids = wl.serving_grids()
    gi = 2
    spec_g, ne = grids[gi]
    h = rt.Grid(spec_g, ne)
    reqs = [f for g, f in wl.serving_requests(2000, 9, [g for g, _ in grids]) if g == gi]
    sizes = [rt.Fan(f).n_rays for f in reqs]
    big = reqs[int(np.argmax(sizes))]
    small = [f for f, n in zip(reqs, sizes) if n <= 2000][:64]
    srv = rt.Server(max_inflight=1, fuse_max_rays=fuse)
    per_launch = []
    for _ in range(rounds):
        fans = [rt.Fan(big)] + [rt.Fan(f) for f in small]
        tickets = [srv.submit(h, f) for f in fans]
        per_launch = [srv.wait(t[0], timeout_s=600.0).batch_size for t in tickets]
    srv.close()
    h.close()
    print(json.dumps({"profile_run": True, "workload": "fused small requests", "rounds": rounds,
                      "large_request_rays": int(max(sizes)), "small_requests": len(small),
                      "small_rays": int(sum(rt.Fan(f).n_rays for f in small)),
                      "requests_per_launch_last_round": per_launch[1:]}), flush=True)


def run_serving(rt, wl, seconds, seed=9, slots=8, fuse=16384):
    """Serving form: a Poisson stream of uneven fan requests (1..100k rays,
    ionogram-synthesis and OTHR-registration shapes) over four resident grids
    (21x21x61 .. 181x361x301), through the continuous-batching server.  The
    saturated throughput of the same request mix is measured first (all
    requests submitted at once), one 96-request list served three ways: one
    launch per request, the persistent kernel, and fusion of requests of at
    most `fuse` rays; offered loads of 10 %, 50 % and 90 % of the first
    follow, each for `seconds` of arrivals, served without and with fusion
    (same requests, same arrival times).  Latency = submit -> records in the
    caller's host buffer."""
    grids = wl.serving_grids()
    handles = [rt.Grid(g, ne) for g, ne in grids]
    specs = [g for g, _ in grids]
    stream_reqs = iter(wl.serving_requests(3 * 16 + 96 + 3 * 2000, seed, specs))

    def server(**kw):
        return rt.Server(max_inflight=slots, mem_reserve_bytes=1 << 30, **kw)

    def run(srv, reqs, arrivals):
        fans = [rt.Fan(f) for _, f in reqs]
        done = [None] * len(reqs)
        tickets = [None] * len(reqs)
        t_sub = [0.0] * len(reqs)
        ready = threading.Semaphore(0)

        def waiter():
            for i in range(len(reqs)):
                ready.acquire()
                done[i] = srv.wait(tickets[i][0], timeout_s=600.0)

        th = threading.Thread(target=waiter)
        th.start()
        t0 = time.perf_counter()
        for i, (gi, _) in enumerate(reqs):
            dt = t0 + arrivals[i] - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            t_sub[i] = time.perf_counter() - t0
            tickets[i] = srv.submit(handles[gi], fans[i])
            ready.release()
        th.join()
        lat = np.array([d.total_s for d in done])
        ends = np.array(t_sub) + lat
        rays = sum(f.n_rays for f in fans)
        evals = sum(int(t[1]["n_evals"].sum()) for t in tickets)
        bad = sum(int(d.status != rt.RT_OK) for d in done)
        span = float(ends.max())  # first submit at t = 0
        fp32_peak = SMS * FP32_LANES_PER_SM * 2 * 2070e6
        return {"requests": len(reqs), "rays": rays, "rays_per_s": rays / span,
                "stage_evals_per_s": evals / span,
                "fp32_roofline_frac": evals * FLOP_PER_EVAL["mixed"] / span / fp32_peak,
                "latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3), "p99": float(np.percentile(lat, 99) * 1e3)},
                "queue_ms_p50": float(np.percentile([d.queue_s for d in done], 50) * 1e3),
                "requests_per_launch_mean": float(np.mean([d.batch_size for d in done])),
                "failed": bad}

    def take(k):
        return [next(stream_reqs) for _ in range(k)]

    plain, persistent, fused = server(), server(cfg=rt.launch_config(kernel=rt.RT_KERNEL_PERSISTENT)), \
        server(fuse_max_rays=fuse)
    for srv in (plain, persistent, fused):
        run(srv, take(16), np.zeros(16))  # warm-up: every grid and kernel variant touched
    sat_reqs = take(96)
    sat = run(plain, sat_reqs, np.zeros(96))
    sat_p = run(persistent, sat_reqs, np.zeros(96))
    sat_f = run(fused, sat_reqs, np.zeros(96))
    persistent.close()
    peak = sat["rays_per_s"]
    mean_rays = wl.serving_mean_rays()
    out = {"grids": [list(g.shape) for g in specs], "max_inflight": slots, "fuse_max_rays": fuse,
           "saturated": sat, "saturated_persistent_kernel": sat_p, "saturated_fused": sat_f,
           "small_fans": small_fans_compare(rt, wl), "loads": {}, "loads_fused": {}}
    rng = np.random.default_rng(seed + 1)
    for frac in (0.1, 0.5, 0.9):
        rate = frac * peak / mean_rays  # requests per second
        k = int(np.clip(rate * seconds, 40, 2000))
        arrivals = np.cumsum(rng.exponential(1.0 / rate, k))
        reqs = take(k)
        key = "%d%%" % round(frac * 100)
        out["loads"][key] = dict(run(plain, reqs, arrivals), offered_rays_per_s=frac * peak)
        out["loads_fused"][key] = dict(run(fused, reqs, arrivals), offered_rays_per_s=frac * peak)
    plain.close()
    fused.close()
    for h in handles:
        h.close()
    return out


def main():
    faulthandler.enable()  # a native crash prints every thread's Python stack
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
