"""Benchmark: RK4 particle-steps/s of the 3-D FP32 advection step on a global
1/4-degree grid (1440 x 720 x 50 levels, 30 daily snapshots of U, V, W, two
bracketing snapshots sampled per stage, periodic zonal boundary, deletion out
of the depth/latitude range), 10 million particles in the upper 1000 m, dt 30
minutes for 30 days (1440 steps).

One bench step = one full execute of that workload from the seeded start
state.  `value` times the steps with the field and particles resident in HBM;
`e2e` runs the same workload through the C ABI from host buffers (snapshots
streamed host-to-device during the run, particles uploaded and results read
back inside the timed region).  `--impl reference` times the FP64 CPU oracle on
a bounded sample of the same workload instead.

Launch: python bench.py [--steps K] [--warmup W]   (N > 1 under torchrun)
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DAY = 86400.0
ALGO_BYTES_PER_STEP = 810.0      # 3-D FP32 RK4: 768 B of field gathers + 42 B of state
ALGO_FLOPS_PER_STEP = 450.0
METRIC = "RK4 particle-steps/s on 1 GB300, chosen form vs plain FP32 at ≤1e-3-cell error"
UNIT = "particle-steps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--particles", type=int, default=10_000_000)
    ap.add_argument("--days", type=float, default=30.0)
    ap.add_argument("--snapshots", type=int, default=30,
                    help="daily snapshots in the periodic field (30 = the workload)")
    ap.add_argument("--block", type=int, default=128)
    ap.add_argument("--resort-steps", type=int, default=1440,
                    help="Morton re-sort before the first launch of each execute and every this "
                         "many steps (0: never); 1440: one sort per 30-day run of the 3-D "
                         "workload (re-sorting every 288 steps as well measured 1.2 %% slower)")
    ap.add_argument("--chunk-steps", type=int, default=1440,
                    help="at most this many steps per kernel launch (1440: the 30-day run of the "
                         "3-D workload in one launch where nothing else ends it; 288: 0.8 %% slower)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-ring", type=int, default=16,
                    help="snapshot ring slots of the end-to-end leg (4: two in use + the next; "
                         "8: three-day launches; 16: six-day launches)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-mlp", action="store_true",
                    help="skip the surrogate network's inference timing in the 3-D line")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--workload", default="3d",
                    choices=["3d", "precision", "batch", "surrogate", "example", "rkf45", "mlp"],
                    help="3d: the FP32 3-D workload (default); precision: 2-D 1/12 deg "
                         "cell-index + FP16/BF16 form against plain FP32; batch: 256 "
                         "releases in one persistent launch per day, graph-captured; "
                         "example: the worked example's backward two-phase run with "
                         "sampled temperature and daily indexed output; rkf45: adaptive "
                         "RKF45 on the 3-D workload; mlp: the surrogate network's "
                         "inference on --mlp-rows feature rows, three engines")
    ap.add_argument("--mlp-rows", type=int, default=10_000_000)
    ap.add_argument("--rkf45-tol", type=float, default=10.0, help="metres per step")
    ap.add_argument("--batch-scale", type=float, default=1.0,
                    help="shrink every release of the batch workload (tests)")
    ap.add_argument("--train-segments", type=int, default=20_000_000)
    ap.add_argument("--train-steps", type=int, default=20000)
    ap.add_argument("--sur-days", type=float, default=180.0)
    ap.add_argument("--engine", default="tcgen05", choices=["tcgen05", "mma.sync"],
                    help="tensor-core engine of the surrogate's products (tcgen05: fused "
                         "inference forward, tcgen05 training products)")
    ap.add_argument("--storage", default="f16", choices=["f16", "bf16"])
    return ap.parse_args()


def reduce_over_ranks(elapsed_ms, particle_steps, device):
    """Whole-job timing under torchrun: the maximum of the ranks' timed regions
    and the sum of their particle-steps.  Each rank advects its own particles
    (weak scaling, no data-path collective); this reduction is the only
    collective of the run."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(elapsed_ms), float(particle_steps)
    t = torch.tensor([float(elapsed_ms), float(particle_steps)], device=device,
                     dtype=torch.float64)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = t.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm[1])


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            for k in ("hbm_gbs", "hbm_GBps", "hbm"):
                if k in d:
                    return float(d[k]), "measured"
        except Exception:
            pass
    return 6800.0, "fallback"


def kernel_hash():
    h = hashlib.sha256()
    for f in ("advect_common.cuh", "advect_plain.cuh", "advect_f32.cu", "pg_device.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1707_05163_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def captured_traffic():
    """Per-particle-step DRAM and L2 bytes of the advection kernel from a
    committed ncu capture, or None when the capture was taken on another
    version of the kernel source."""
    p = os.path.join(ROOT, "profiles", "advect_f32_3d_traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
        if d.get("kernel_hash") == kernel_hash():
            return d
    except Exception:
        pass
    return None


def l2_read_peak(lib):
    """Measured L2 read bandwidth (GB/s) of this GPU: the library's probe, a
    32 MiB L2-resident buffer read with coalesced 16-byte loads that bypass
    L1, best of 10 launches."""
    import ctypes as C
    g = C.c_double()
    if lib.pg_measure_l2_read(32 << 20, 10, C.byref(g), None) != 0:
        return None
    return g.value


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, gpu_index):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={gpu_index}",
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 8:
                rows.append(parts)
        if not rows:
            return None
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(mx)) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def bf16_burst_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(p))["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


def mlp_forward_leg(pg, torch, dev, x=None, rows=10_000_000, engines=(("tcgen05_fused", 1),),
                    net=None, reps=5):
    """Inference throughput of the surrogate network (37 inputs padded to 64,
    4 hidden layers of 256, 3 outputs padded to 64: 2 * (64*256 + 3*256*256 +
    256*64) FLOP per row) on `rows` feature rows resident on the device, input
    packing included; CUDA events on the current stream, best of `reps`, one
    warm-up.  Random-initialised weights unless a trained `net` is given."""
    flop_row = 2.0 * (64 * 256 + 3 * 256 * 256 + 256 * 64)
    if net is None:
        net = pg.MLP(37, 256, 4, 3, seed=5)
    if x is None:
        g = torch.Generator(device=dev)
        g.manual_seed(7)
        x = torch.randn(rows, 37, device=dev, generator=g)
    peak, kind = bf16_burst_peak()
    out = {}
    for name, flag in engines:
        net.set_engine(flag)
        net.forward(x)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        best = float("inf")
        for _ in range(reps):
            e0.record()
            net.forward(x)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        tf = flop_row * x.shape[0] / (best * 1e-3) / 1e12
        out[name] = {"ms_per_10M_rows": best * 1e7 / x.shape[0], "TFLOPs": tf,
                     "frac_of_bf16_peak": tf / peak, "peak_TFLOPs": peak, "peak_source": kind}
    return out


def make_field_host_bases(gf):
    return [gf.base2d(s) for s in range(len(gf.times))]


def oracle_baseline(gf, host_field, lon, lat, dep, days, seconds_budget):
    """The FP64 oracle on a bounded sample of the workload, on this host's cores."""
    import oracle as O
    cores = len(os.sched_getaffinity(0))
    f = O.Field(gf.lon, gf.lat, gf.depth, gf.times, host_field, 1, True, gf.period)
    k = O.Kernel(O.RK4)

    def run(n, steps_days):
        st = [np.array(lon[:n], np.float64), np.array(lat[:n], np.float64),
              np.array(dep[:n], np.float64), np.zeros(n), np.arange(n, dtype=np.uint64),
              np.zeros(n, np.uint32), np.zeros(n, np.uint8)]
        t0 = time.perf_counter()
        done = O.run(f, k, *st, 1800.0, steps_days * DAY, steps_days * DAY, nthreads=cores)
        return done, time.perf_counter() - t0

    n0 = 32 * cores
    done, dt = run(n0, days)
    n = int(min(len(lon), max(n0, n0 * seconds_budget / max(dt, 1e-3))))
    done, dt = run(n, days)
    return {"value": done / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {n} of the workload's particles, full {days:g}-day horizon, "
                      f"{done} particle-steps in {dt:.1f} s"}, done, dt


def build_fieldset_device(pg, gf, torch, dev, bases, host_field=None):
    """All snapshots resident: each slab built on the device (float32 of the
    FP64 product base x profile, the same values the host generator makes)."""
    fs = pg.FieldSet(gf.lon, gf.lat, gf.depth, mesh="spherical", periodic_lon=True,
                     nfields=gf.nfields, storage="f32")
    fs.set_times(gf.times, gf.period)
    prof = torch.from_numpy(gf.profiles()).to(dev)
    for s, b in enumerate(bases):
        base = torch.from_numpy(b).to(dev)
        slab = (base[:, None, :, :] * prof[:, :, None, None]).to(torch.float32)
        fs.load_snapshot(s, slab)
        if host_field is not None:
            host_field[s].copy_(slab)
        del slab, base
    torch.cuda.synchronize()
    return fs


def main():
    args = parse()
    rank, world, local = dist_env()
    import torch
    if args.impl == "reference":
        return reference_arm(args, rank, world)
    if args.workload == "precision":
        return precision_workload(args, rank, world, local)
    if args.workload == "batch":
        return batch_workload(args, rank, world, local)
    if args.workload == "surrogate":
        return surrogate_workload(args, rank, world, local)
    if args.workload in ("example", "rkf45"):
        return example_or_rkf45_workload(args, rank, world, local)
    if args.workload == "mlp":
        return mlp_workload(args, rank, world, local)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    import paper_1707_05163_gb300 as pg
    import synth
    pg.load()

    gf = synth.GlobalField(res_deg=0.25, nz=50, nt=args.snapshots, seed=2,
                           period=args.snapshots * DAY)
    bases = make_field_host_bases(gf)
    want_host = (not args.no_e2e) or (rank == 0 and world == 1 and not args.no_cpu)
    host_field = None
    if want_host:
        try:
            host_field = torch.empty((len(gf.times), gf.nfields, gf.nz, gf.ny, gf.nx),
                                     dtype=torch.float32, pin_memory=True)
        except Exception:
            host_field = None
    fs = build_fieldset_device(pg, gf, torch, dev, bases, host_field)

    n = args.particles
    lon, lat, dep = synth.uniform_particles(n, 2 + rank, (0.0, 360.0), (-80.0, 80.0),
                                            (5.0, 1000.0), dtype=np.float32)
    dlon = torch.from_numpy(lon).to(dev)
    dlat = torch.from_numpy(lat).to(dev)
    ddep = torch.from_numpy(dep).to(dev)
    kern = pg.Kernel("rk4")
    runtime = args.days * DAY
    lib = pg.load()
    import ctypes as C

    def one_step(timing=False):
        ps = pg.ParticleSet(fs, dlon, dlat, ddep, pos="f32", seed=0)
        ps.set_tune(args.block, args.resort_steps, args.chunk_steps)
        if timing:
            lib.pg_pset_kernel_timing(ps.h, 1, None, None)
        steps = ps.execute(kern, runtime, 1800.0)
        ms, launches = C.c_double(), C.c_int64()
        if timing:
            lib.pg_pset_kernel_timing(ps.h, -1, C.byref(ms), C.byref(launches))
        ps.destroy()
        return steps, ms.value, launches.value

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    c0 = C.c_int64()
    lib.pg_launch_count(C.byref(c0))
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    total_steps, kern_ms, kern_launches = 0, 0.0, 0
    for _ in range(args.steps):
        s, ms, ln = one_step(timing=True)
        total_steps += s
        kern_ms += ms
        kern_launches += ln
    ev1.record()
    torch.cuda.synchronize()
    elapsed_ms = ev0.elapsed_time(ev1)
    c1 = C.c_int64()
    lib.pg_launch_count(C.byref(c1))
    clk = clocks.stop()
    elapsed_ms, total_all = reduce_over_ranks(elapsed_ms, total_steps, dev)
    value = total_all / (elapsed_ms / 1e3)

    # the field streamed from pinned host memory (4 slots: two snapshots in
    # use plus the next one uploading; 8 slots: three-day launches):
    # device-timed with particles on the device, and end to end through the
    # C ABI from host buffers
    e2e, streamed = None, None
    if not args.no_e2e and host_field is not None:
        streamed = {f"ring{r}": streamed_leg(pg, gf, torch, host_field, lon, lat, dep, kern,
                                             runtime, args, r, False)
                    for r in sorted({4, args.e2e_ring})}
        e2e = streamed_leg(pg, gf, torch, host_field, lon, lat, dep, kern, runtime, args,
                           args.e2e_ring, True)

    output = None
    if not args.no_e2e:
        output = output_leg(pg, fs, torch, dlon, dlat, ddep, kern, runtime, args)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu and host_field is not None:
        cpu, _, _ = oracle_baseline(gf, host_field.numpy(), lon, lat, dep, args.days,
                                    args.cpu_seconds)

    hbm_peak, peak_kind = measured_peaks()
    l2_peak = l2_read_peak(lib) if rank == 0 else None
    avg_launch_s = (kern_ms / 1e3) / max(kern_launches, 1)
    steps_per_launch = total_steps / max(kern_launches, 1)
    kernel_rate = steps_per_launch / avg_launch_s          # particle-steps/s inside the kernel
    # The kernel keeps each cell's corner values in registers across stages
    # and steps, so it is bound by instruction issue, not by memory: report it
    # against the FP32 FMA peak (SMs x 128 lanes x 2 FLOP x SM clock).
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = (clk or {}).get("sm_max_mhz") or 2070.0
    fp32_peak = sms * 128 * 2 * sm_mhz * 1e6 / 1e12
    achieved = ALGO_FLOPS_PER_STEP * kernel_rate / 1e12
    cap = captured_traffic()
    traffic = cap["dram_bytes_per_particle_step"] * steps_per_launch if cap else None
    l2_view = hbm_view = None
    if cap and cap.get("l2_bytes_per_particle_step") and l2_peak:
        b = cap["l2_bytes_per_particle_step"]
        l2_view = {"bytes_per_particle_step": b, "achieved_GBps": b * kernel_rate / 1e9,
                   "peak_GBps": l2_peak, "frac": b * kernel_rate / 1e9 / l2_peak,
                   "peak_source": "measured live: 32 MiB L2-resident buffer, coalesced "
                                  "ld.global.cg, best of 10 (pg_measure_l2_read)"}
    if cap:
        b = cap["dram_bytes_per_particle_step"]
        hbm_view = {"bytes_per_particle_step": b, "achieved_GBps": b * kernel_rate / 1e9,
                    "peak_GBps": hbm_peak, "frac": b * kernel_rate / 1e9 / hbm_peak,
                    "peak_source": peak_kind}
    # instruction issue: each SM issues at most one warp instruction per cycle
    # on each of its 4 schedulers; the kernel's count per warp-step (32
    # particle-steps) comes from the same committed capture as the bytes
    issue_view = None
    if cap and cap.get("warp_instructions_per_warp_step"):
        ipps = cap["warp_instructions_per_warp_step"] / 32.0
        ipk = sms * 4 * sm_mhz * 1e6
        issue_view = {"warp_instructions_per_particle_step": ipps,
                      "achieved_warp_inst_per_s": ipps * kernel_rate, "peak_warp_inst_per_s": ipk,
                      "frac": ipps * kernel_rate / ipk,
                      "peak_source": f"derived: {sms} SMs x 4 schedulers x 1 warp instruction "
                                     "per cycle x max SM clock"}
    gather_gbs = ALGO_BYTES_PER_STEP * kernel_rate / 1e9
    mlp = None
    if rank == 0 and not args.no_mlp:
        mlp = mlp_forward_leg(pg, torch, dev)["tcgen05_fused"]
        mlp["rows"] = 10_000_000
        mlp["network"] = ("surrogate MLP 37-256x4-3, random-initialised BF16 weights, fused "
                          "tcgen05 inference kernel (input packing included)")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded k^-3 random streamfunction field, uniform particles)",
        "config": {"workload": "3-D FP32 RK4, global 1/4 deg 1440x720x50, 30 daily snapshots "
                               "(periodic), 10M particles upper 1000 m, dt 30 min, 30 days",
                   "particles_per_gpu": n, "days": args.days, "dt_s": 1800.0,
                   "block": args.block, "resort_steps": args.resort_steps,
                   "chunk_steps": args.chunk_steps, "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (24.9 GB field, 10M-particle state)"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak,
                     "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": traffic,
                     "alu_frac": achieved / fp32_peak,
                     "l2_frac": l2_view["frac"] if l2_view else None,
                     "hbm_frac": hbm_view["frac"] if hbm_view else None,
                     "issue_frac": issue_view["frac"] if issue_view else None,
                     "peak_source": f"derived: {sms} SMs x 128 FP32 lanes x 2 FLOP x max SM clock",
                     "kernel": "advect_plain_kernel<float, float, 3, true, GEO_SPH_PER>",
                     "algorithmic_flops_per_particle_step": ALGO_FLOPS_PER_STEP,
                     "avg_launch_ms": avg_launch_s * 1e3, "launches": kern_launches,
                     "l2": l2_view, "hbm": hbm_view, "issue": issue_view,
                     "l2_read_peak_GBps": l2_peak,
                     "traffic_capture": cap.get("captured") if cap else None,
                     "gather_view": {"algorithmic_bytes_per_particle_step": ALGO_BYTES_PER_STEP,
                                     "effective_GBps": gather_gbs,
                                     "meaning": "the corner values the definition gathers at "
                                                "every stage, 768 B + 42 B of state; the "
                                                "kernel keeps a cell's corners in registers, "
                                                "so its L2 and DRAM traffic (l2, hbm) is far "
                                                "below this"}},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "streamed": streamed,
        "output": output,
        "surrogate_mlp_forward": mlp,
        "gpu_launches": int(c1.value - c0.value),
        "clocks": clk,
        "particle_steps": total_all,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def output_leg(pg, fs, torch, dlon, dlat, ddep, kern, runtime, args):
    """Trajectory output at scale (the ParticleFile of Sect. 3): the same
    resident run with daily output in the indexed form through the pinned
    ring (rows packed on the GPU, copied on a side stream, handed to a hook
    that only counts them), against the run without output.  Best of two,
    device-timed around the execute."""
    import ctypes as C
    lib = pg.load()
    rows = [0, 0]

    def hook(user, rp):
        rows[0] += rp.contents.n
        rows[1] += 1
        return 0
    cb = pg._native.RECORD_CB(hook)
    res = {}
    for mode in ("none", "indexed_daily"):
        best = None
        for _ in range(2):
            ps = pg.ParticleSet(fs, dlon, dlat, ddep, pos="f32", seed=0)
            ps.set_tune(args.block, args.resort_steps, args.chunk_steps)
            rows[0] = rows[1] = 0
            steps = C.c_int64()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            ev0.record()
            if mode == "none":
                r = lib.pg_execute(ps.h, kern.h, runtime, 1800.0, 0.0, pg._native.OUTPUT_CB(),
                                   None, None, C.byref(steps))
            else:
                r = lib.pg_execute_records(ps.h, kern.h, runtime, 1800.0, DAY, 1, cb, None, None,
                                           C.byref(steps))
            ev1.record()
            torch.cuda.synchronize()
            assert r == 0, lib.pg_last_error()
            ms = ev0.elapsed_time(ev1)
            ps.destroy()
            if best is None or ms < best[0]:
                best = (ms, steps.value, rows[0], rows[1])
        res[mode] = {"ms": best[0], "particle_steps_per_s": best[1] / (best[0] / 1e3),
                     "rows": best[2], "outputs": best[3]}
    n = len(dlon)
    res["ring_bytes_per_output"] = n * (8 * 5 + 1)
    res["overhead"] = res["indexed_daily"]["ms"] / res["none"]["ms"] - 1.0
    return res


def streamed_leg(pg, gf, torch, host_field, lon, lat, dep, kern, runtime, args, ring,
                 from_host):
    """The workload with its snapshots streamed from pinned host memory
    through a ring of `ring` device slots (4: two snapshots in use by a
    launch, one for steps that reach past it, the next uploading; launches
    end at the next snapshot time; larger rings: launches of (ring - 4) / 2
    + 1 days, the spare slots prefetching).  from_host: particles uploaded from
    pinned FP64 host arrays and the final state read back into them, all
    inside the timed region (the end-to-end number); otherwise particles
    start on the device and only the execute is timed (CUDA events).
    Returns the best of two runs with its breakdown."""
    import ctypes as C
    n = len(lon)
    fs = pg.FieldSet(gf.lon, gf.lat, gf.depth, mesh="spherical", periodic_lon=True,
                     nfields=gf.nfields, storage="f32")
    fs.set_times(gf.times, gf.period)
    fs.set_ring(ring)
    fs.stream([host_field[s] for s in range(len(gf.times))])
    if from_host:
        src = [torch.from_numpy(np.asarray(a, np.float64)).pin_memory() for a in (lon, lat, dep)]
        out = {k: torch.empty(n, dtype=torch.float64).pin_memory() for k in ("lon", "lat", "depth")}
        ost = torch.empty(n, dtype=torch.uint8).pin_memory()
    else:
        src = [torch.from_numpy(a).cuda() for a in (lon, lat, dep)]
    lib = pg.load()
    best = None
    for rep in range(2):
        lib.pg_fieldset_stats(fs.h, 1, None, None)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        ev[0].record()
        ps = pg.ParticleSet(fs, src[0], src[1], src[2], pos="f32", seed=0)
        ev[1].record()
        ps.set_tune(args.block, args.resort_steps, args.chunk_steps)
        lib.pg_pset_kernel_timing(ps.h, 1, None, None)
        steps = ps.execute(kern, runtime, 1800.0)
        ev[2].record()
        if from_host:
            ps.get_into(lon=out["lon"], lat=out["lat"], depth=out["depth"], status=ost)
        ev[3].record()
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
        kms, kl = C.c_double(), C.c_int64()
        lib.pg_pset_kernel_timing(ps.h, -1, C.byref(kms), C.byref(kl))
        ps.destroy()
        ups, ub = C.c_int64(), C.c_int64()
        lib.pg_fieldset_stats(fs.h, 1, C.byref(ups), C.byref(ub))
        ex_ms = ev[1].elapsed_time(ev[2])
        rec = {"wall_s": wall, "steps": steps,
               "particles_h2d_ms": ev[0].elapsed_time(ev[1]), "execute_ms": ex_ms,
               "advection_kernels_ms": kms.value, "launches": kl.value,
               "execute_other_ms": ex_ms - kms.value,
               "results_d2h_ms": ev[2].elapsed_time(ev[3]),
               "snapshot_uploads": ups.value, "snapshot_h2d_bytes": ub.value}
        key = wall if from_host else ex_ms
        if best is None or key < best[0]:
            best = (key, rec)
    fs.destroy()
    rec = best[1]
    rec["ring"] = ring
    rec["note"] = ("execute_other_ms = execute minus its advection kernels: re-sorts, waits "
                   "for snapshot uploads, launch gaps")
    if from_host:
        h2d = rec["snapshot_h2d_bytes"] + n * 3 * 8        # snapshots + FP64 positions
        d2h = n * (3 * 8 + 1)
        return {"value": rec["steps"] / rec["wall_s"], "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "seconds": rec["wall_s"], "breakdown": rec}
    rec["value"] = rec["steps"] / (rec["execute_ms"] / 1e3)
    rec["unit"] = UNIT
    return rec


def reference_arm(args, rank, world):
    """The FP64 CPU oracle as the reference arm, on a bounded sample per step."""
    if rank != 0:
        return
    import synth
    gf = synth.GlobalField(res_deg=0.25, nz=50, nt=30, seed=2)
    field = np.empty((len(gf.times), gf.nfields, gf.nz, gf.ny, gf.nx), dtype=np.float32)
    for s in range(len(gf.times)):
        field[s] = gf.slab(s)
    lon, lat, dep = synth.uniform_particles(args.particles, 2, (0.0, 360.0), (-80.0, 80.0),
                                            (5.0, 1000.0), dtype=np.float32)
    budget = max(2.0, 120.0 / max(args.steps + args.warmup, 1))
    cpu, done, dt = None, 0, 0.0
    for i in range(args.warmup + args.steps):
        c, d, t = oracle_baseline(gf, field, lon, lat, dep, args.days, budget)
        if i >= args.warmup:
            done += d
            dt += t
            cpu = c
    value = done / dt
    cpu["value"] = value
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": "3-D RK4, global 1/4 deg 1440x720x50, 30 daily "
                                                    "snapshots, dt 30 min, 30 days (oracle sample)"},
        "cpu_baseline": cpu,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def example_or_rkf45_workload(args, rank, world, local):
    """example: the paper's worked example (Sect. 3) at scale on the 3-D
    1/4-degree field with a synthetic temperature field: particles released
    around 17.3 E, 34.7 S at 2440 m are run backward in time with 5-minute
    RK4 steps; they rise at 200 m/day to their 50 m dwelling depth, live
    there 30 days (age), sample temperature every step, and go to a daily
    indexed trajectory output through the pinned ring.  rkf45: the 3-D
    workload's particles and horizon with adaptive RKF45 steps (tolerance
    --rkf45-tol metres, steps between 60 s and 2 h).  Each is compared with
    plain FP32 RK4 at dt 30 min on the same particles."""
    import ctypes as C
    import torch
    import paper_1707_05163_gb300 as pg
    import synth
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    gf = synth.GlobalField(res_deg=0.25, nz=50, nt=30, seed=2, period=30 * DAY)
    fs = build_fieldset_device(pg, gf, torch, dev, make_field_host_bases(gf))
    lib = pg.load()
    example = args.workload == "example"
    if example:
        n = args.particles if args.particles != 10_000_000 else 1_000_000
        rng = np.random.default_rng(11)
        lon = (17.3 + rng.uniform(-2.0, 2.0, n)).astype(np.float32)
        lat = (-34.7 + rng.uniform(-2.0, 2.0, n)).astype(np.float32)
        dep = np.full(n, 2440.0, np.float32)
        fs.add_scalar("temperature")
        base = synth.temperature_base(gf.lon, gf.lat, gf.depth, seed=4, dtype=np.float32)
        for s in range(len(gf.times)):
            fs.load_scalar(0, s, torch.from_numpy(synth.temperature_at(base, gf.times[s],
                                                                       gf.period)).to(dev))
        del base
        fs.add_constant("w_sink", 200.0 / DAY)
        fs.add_constant("dwelling_depth", 50.0)
        fs.add_constant("max_age", 30 * DAY)
        kern = pg.Kernel("rk4", ("settle", "age", "sample"), w_sink=None)
        t0, runtime, dt = 45 * DAY, 45 * DAY, -300.0
    else:
        n = args.particles
        lon, lat, dep = synth.uniform_particles(n, 2, (0.0, 360.0), (-80.0, 80.0),
                                                (5.0, 1000.0), dtype=np.float32)
        fs.add_constant("rkf45_tol", args.rkf45_tol)
        fs.add_constant("rkf45_min_dt", 60.0)
        fs.add_constant("rkf45_max_dt", 7200.0)
        kern = pg.Kernel("rkf45")
        t0, runtime, dt = 0.0, args.days * DAY, 1800.0
    dl, da, dd = (torch.from_numpy(a).to(dev) for a in (lon, lat, dep))
    rows = [0, 0]

    def hook(user, rp):
        rows[0] += rp.contents.n
        rows[1] += 1
        return 0
    cb = pg._native.RECORD_CB(hook)

    def run(k, step_dt, timed):
        ps = pg.ParticleSet(fs, dl, da, dd, t0=t0 if example else 0.0, pos="f32", seed=1)
        ps.set_tune(args.block, args.resort_steps, args.chunk_steps)
        lib.pg_pset_kernel_timing(ps.h, 1, None, None)
        rows[0] = rows[1] = 0
        steps = C.c_int64()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record()
        if example and k is kern:
            r = lib.pg_execute_records(ps.h, k.h, runtime, step_dt, DAY, 1, cb, None, None,
                                       C.byref(steps))
        else:
            r = lib.pg_execute(ps.h, k.h, runtime, step_dt, 0.0, pg._native.OUTPUT_CB(), None,
                               None, C.byref(steps))
        ev1.record()
        torch.cuda.synchronize()
        assert r == 0, lib.pg_last_error()
        kms, kl = C.c_double(), C.c_int64()
        lib.pg_pset_kernel_timing(ps.h, -1, C.byref(kms), C.byref(kl))
        g = ps.get() if timed else None
        v = ps.get_variables() if (timed and example) else None
        ps.destroy()
        return steps.value, ev0.elapsed_time(ev1), kms.value, g, v, tuple(rows)

    for _ in range(max(1, args.warmup)):
        run(kern, dt, False)
    clocks = ClockSampler(local)
    best = None
    for _ in range(max(1, args.steps)):
        r = run(kern, dt, True)
        if best is None or r[1] < best[1]:
            best = r
    clk = clocks.stop()
    steps, ms, kms, g, v, rec = best
    plain = run(pg.Kernel("rk4"), -1800.0 if example else 1800.0, not example)
    line = {
        "metric": METRIC, "value": steps / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded k^-3 random streamfunction field, synthetic temperature)",
        "config": {"workload": ("worked example, backward: %d particles at 2440 m near 17.3E "
                                "34.7S, RK4 dt 5 min, rise at 200 m/day to 50 m, 30-day "
                                "lifespan, temperature sampled, daily indexed output, 3-D "
                                "1/4 deg field" % n) if example else
                               ("RKF45 on the 3-D workload: %d particles, %g days, tol %g m, "
                                "steps 60 s to 2 h" % (n, args.days, args.rkf45_tol)),
                   "block": args.block, "resort_steps": args.resort_steps,
                   "chunk_steps": args.chunk_steps},
        "particle_steps": steps, "advection_kernel_ms": kms,
        "plain_fp32_rk4_30min": {"particle_steps": plain[0], "ms": plain[1],
                                 "particle_steps_per_s": plain[0] / (plain[1] / 1e3)},
        "clocks": clk,
    }
    if example:
        st = g["status"]
        line["example"] = {"output_rows": rec[0], "outputs": rec[1],
                           "deleted_by_age": int((st == 4).sum()), "alive": int((st == 0).sum()),
                           "out_of_domain": int(((st == 1) | (st == 2)).sum()),
                           "mean_lifespan_temperature_at_death_degC":
                               float(np.nanmean(v["vars"][0][st == 4])) if (st == 4).any() else None}
    else:
        # accuracy at equal cost: both against RK4 with 5-minute steps
        ref = run(pg.Kernel("rk4"), 300.0, True)[3]

        def err_cells(x):
            ok = (x["status"] == 0) & (ref["status"] == 0)
            dlon = (x["lon"] - ref["lon"] + 180.0) % 360.0 - 180.0
            e = np.maximum(np.abs(dlon), np.abs(x["lat"] - ref["lat"]))[ok] / 0.25
            return {"mean_cells": float(e.mean()), "median_cells": float(np.median(e)),
                    "p99_cells": float(np.percentile(e, 99))}
        alive = g["status"] == 0
        line["rkf45"] = {"mean_steps_per_particle": float(g["step"][alive].mean()),
                         "min_steps": int(g["step"][alive].min()),
                         "max_steps": int(g["step"][alive].max()),
                         "fixed_rk4_steps_per_particle": args.days * DAY / 1800.0,
                         "error_vs_rk4_5min": err_cells(g),
                         "rk4_30min_error_vs_rk4_5min": err_cells(plain[3])}
    print(json.dumps(line), flush=True)


def mlp_workload(args, rank, world, local):
    """The surrogate network alone (37 inputs, 4 hidden layers of 256, 3
    outputs; random-initialised BF16 weights): inference on --mlp-rows
    Gaussian feature rows resident on the device, for the fused tcgen05
    kernel, the layer-by-layer tcgen05 products and the mma.sync products.
    `value` is the fused kernel's rows per second; one process, replicas
    only (the rows are independent)."""
    import ctypes as C
    import torch
    import paper_1707_05163_gb300 as pg
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lib = pg.load()
    c0, c1 = C.c_int64(), C.c_int64()
    lib.pg_launch_count(C.byref(c0))
    engines = mlp_forward_leg(pg, torch, dev, rows=args.mlp_rows, reps=max(args.steps, 1),
                              engines=(("tcgen05_fused", 1), ("tcgen05_layer_by_layer", 2),
                                       ("mma.sync", 0)))
    lib.pg_launch_count(C.byref(c1))
    launches = int(c1.value - c0.value)
    f = engines["tcgen05_fused"]
    rows_per_s = 1e7 / (f["ms_per_10M_rows"] * 1e-3)
    line = {
        "metric": "surrogate MLP inference rows/s", "value": rows_per_s, "unit": "rows/s",
        "n_gpus": 1, "steps": args.steps, "warmup": 1, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16 (fp32 accumulate)",
        "data": "synthetic (Gaussian feature rows, random-initialised weights)",
        "config": {"workload": f"surrogate MLP 37-256x4-3 inference, {args.mlp_rows} rows",
                   "l2": "inputs larger than L2 (1.48 GB of features at 10M rows)"},
        "roofline": {"bound": "tensor", "achieved": f["TFLOPs"], "peak": f["peak_TFLOPs"],
                     "unit": "TFLOP/s", "frac": f["frac_of_bf16_peak"], "traffic": None,
                     "kernel": "mlp_fused_kernel",
                     "algorithmic_flops_per_row": 2.0 * (64 * 256 + 3 * 256 * 256 + 256 * 64),
                     "peak_source": f["peak_source"] + " bf16 burst"},
        "engines": engines, "gpu_launches": launches,
    }
    print(json.dumps(line), flush=True)


def surrogate_workload(args, rank, world, local):
    """Learned-surrogate form: an MLP (37 inputs incl. a 4x4x2 U/V stencil, 4
    hidden layers of 256, GELU, BF16 weights, FP32 accumulation) trained with
    the library's kernels on RK4 24 h segments generated on the GPU over the
    3-D 1/4-degree field (30-day periodic), then run for 10M particles over
    180 days with an RK4 check every 5 network steps and RK4 fallback above
    the threshold.  Compared with plain FP32 RK4 on the same particles."""
    import torch
    import paper_1707_05163_gb300 as pg
    from paper_1707_05163_gb300 import surrogate as S
    import synth
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    gf = synth.GlobalField(res_deg=0.25, nz=50, nt=30, seed=2)
    fs = build_fieldset_device(pg, gf, torch, dev, make_field_host_bases(gf))
    t0 = time.perf_counter()
    x, y = S.make_segments(fs, args.train_segments, seed=5, groups=60, period=gf.period)
    t_data = time.perf_counter() - t0
    xv, yv = S.make_segments(fs, 1_000_000, seed=6, groups=20, period=gf.period)
    net = pg.MLP(37, 256, 4, 3, seed=5)
    net.set_engine(args.engine == "tcgen05")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = S.train(net, x, y, steps=args.train_steps, batch=16384, lr=1e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del x, y
    # forward throughput of the two tensor-core engines on 10M feature rows
    # (padded network: 2 * (64*256 + 3*256*256 + 256*64) FLOP per row)
    xb = xv.repeat((10_000_000 + xv.shape[0] - 1) // xv.shape[0], 1)[:10_000_000].contiguous()
    engines = mlp_forward_leg(pg, torch, dev, x=xb, net=net,
                              engines=(("mma.sync", 0), ("tcgen05_layer_by_layer", 2),
                                       ("tcgen05_fused", 1)))
    del xb
    net.set_engine(args.engine == "tcgen05")
    pred = net.forward(xv)
    err = (pred[:, :2] - yv[:, :2]).abs().max(dim=1).values.cpu().numpy()
    held = {"mean_cells": float(err.mean()), "median_cells": float(np.median(err)),
            "within_1e-3": float((err <= 1e-3).mean()), "within_1e-2": float((err <= 1e-2).mean()),
            "within_1e-1": float((err <= 1e-1).mean())}
    n = args.particles
    nsteps = int(round(args.sur_days))
    lon, lat, dep = synth.uniform_particles(n, 7, (0.0, 360.0), (-80.0, 80.0), (5.0, 1000.0),
                                            dtype=np.float32)
    dl, da, dd = (torch.from_numpy(a).to(dev) for a in (lon, lat, dep))
    K = pg.Kernel("rk4")
    # plain FP32 RK4 over the same horizon
    ref = pg.ParticleSet(fs, dl, da, dd, pos="f32")
    ref.set_tune(args.block, args.resort_steps, 48)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rk_steps = ref.execute(K, nsteps * DAY, 1800.0)
    torch.cuda.synchronize()
    t_rk = time.perf_counter() - t0
    g_ref = ref.get()
    ref.destroy()
    runs = {}
    for thr in (1e-3, 1e-2, 1e-1):
        ps = pg.ParticleSet(fs, dl, da, dd, pos="f32")
        ps.set_tune(args.block, args.resort_steps, 48)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = pg.surrogate_run(ps, net, K, nsteps=nsteps, check_every=5, threshold=thr)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        g = ps.get()
        ok = (g["status"] == 0) & (g_ref["status"] == 0)
        dlon = (g["lon"] - g_ref["lon"] + 180.0) % 360.0 - 180.0
        e = np.maximum(np.abs(dlon), np.abs(g["lat"] - g_ref["lat"]))[ok] / 0.25
        runs[f"{thr:g}"] = {"seconds": dt, "speedup_vs_plain_rk4": t_rk / dt,
                            "equivalent_rate": rk_steps / dt,
                            "rejected_fraction": st["rejected"] / max(1, n * (nsteps // 5)),
                            "mean_check_error_cells": st["error_sum"] / max(1, st["checked"]),
                            "final_mean_error_vs_rk4_cells": float(e.mean()) if e.size else None,
                            "network_seconds": st["seconds_network"],
                            "rk4_seconds": st["seconds_rk4"]}
        ps.destroy()
    main = runs["0.001"]
    line = {
        "metric": METRIC, "value": main["equivalent_rate"], "unit": UNIT, "n_gpus": 1,
        "steps": 1, "warmup": 0, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16 MLP (fp32 accumulate) + f32 RK4 check",
        "data": "synthetic (seeded k^-3 random streamfunction field, uniform particles)",
        "config": {"workload": f"surrogate: MLP 37-256x4-3 trained on {args.train_segments} RK4 "
                               f"24 h segments, {n} particles x {nsteps} days, RK4 check every 5 "
                               "steps, fallback above 1e-3 cell, 3-D 1/4 deg field",
                   "engine": args.engine,
                   "value": "equivalent RK4 particle-steps/s (48 steps of 30 min per day)"},
        "plain_fp32_rk4_rate": rk_steps / t_rk,
        "speedup_vs_plain_fp32": main["speedup_vs_plain_rk4"],
        "thresholds": runs, "held_out_24h_error": held, "mlp_forward": engines,
        "training": {"segments_seconds": t_data, "train_seconds": t_train,
                     "steps": args.train_steps, "first_loss": losses[0], "last_loss": losses[-1]},
    }
    print(json.dumps(line), flush=True)


def batch_workload(args, rank, world, local):
    """256 releases (log-uniform sizes 1e3-2e6, dt 10 min-2 h snapped to divisors
    of a day, runtime 5-90 days, kernel mix RK4 / RK4 + Brownian K in [1, 100]
    m^2/s / RK4 + sinking w in [1, 100] m/day) over the 3-D 1/4-degree field
    (30-day periodic), one persistent launch per simulated day, the 90-day
    window loop captured in one CUDA graph, block size and re-sort interval
    from the autotuner.  Compared with one execute per release."""
    import torch
    import paper_1707_05163_gb300 as pg
    import synth
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    gf = synth.GlobalField(res_deg=0.25, nz=50, nt=30, seed=2)
    fs = build_fieldset_device(pg, gf, torch, dev, make_field_host_bases(gf))
    rels = synth.batch_releases(count=256, seed=4, scale=args.batch_scale)
    pos = []
    for r, rel in enumerate(rels):
        lo, la, de = synth.uniform_particles(rel.n, rel.seed, (0.0, 360.0), (-80.0, 80.0),
                                             (5.0, 1000.0), dtype=np.float32)
        pos.append([torch.from_numpy(a).to(dev) for a in (lo, la, de)])

    def kernel(rel):
        if rel.kind == 0:
            return pg.Kernel("rk4")
        if rel.kind == 1:
            return pg.Kernel("rk4", ("brownian",), kh=rel.kh)
        return pg.Kernel("rk4", ("sink",), w_sink=rel.w_sink)
    kernels = [kernel(r) for r in rels]
    rts = [r.runtime for r in rels]
    dts = [r.dt for r in rels]

    def make():
        return [pg.ParticleSet(fs, p[0], p[1], p[2], pos="f32", seed=r.seed,
                               id_base=10_000_000 * i) for i, (p, r) in enumerate(zip(pos, rels))]

    cache = os.path.join(tempfile.gettempdir(), "parcels_gb_batch_tune.txt")
    if os.path.exists(cache):
        os.remove(cache)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    ps = make()
    _, used = pg.execute_batch(ps, kernels, rts, dts, tune=None, tune_cache=cache)
    tune_s = time.perf_counter() - t0
    for p in ps:
        p.destroy()
    for _ in range(max(0, args.warmup - 1)):
        ps = make()
        pg.execute_batch(ps, kernels, rts, dts, tune=used)
        for p in ps:
            p.destroy()
    clocks = ClockSampler(local)
    total, ms = 0, 0.0
    for _ in range(args.steps):
        ps = make()
        torch.cuda.synchronize()
        ev0.record()
        s, _ = pg.execute_batch(ps, kernels, rts, dts, tune=used, use_graph=True)
        ev1.record()
        torch.cuda.synchronize()
        ms += ev0.elapsed_time(ev1)
        total += s
        for p in ps:
            p.destroy()
    clk = clocks.stop()
    value = total / (ms / 1e3)
    # the same releases, one execute per release, one after the other
    ps = make()
    torch.cuda.synchronize()
    ev0.record()
    seq = 0
    for p, k, rt, dt in zip(ps, kernels, rts, dts):
        p.set_tune(used[0], 0, 48)
        seq += p.execute(k, rt, dt)
    ev1.record()
    torch.cuda.synchronize()
    seq_rate = seq / (ev0.elapsed_time(ev1) / 1e3)
    n = sum(r.n for r in rels)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded k^-3 random streamfunction field, uniform particles)",
        "config": {"workload": f"batched: 256 releases, {n} particles, dt 600-7200 s, runtime "
                               "5-90 days, kernel mix, 3-D 1/4 deg field (30-day periodic), "
                               "one persistent launch per day in one CUDA graph",
                   "timed": "the batched execute calls (CUDA events); particle-set creation "
                            "between them is not timed",
                   "autotuned": {"block": used[0], "resort_every_days": used[1],
                                 "tuning_seconds": tune_s}},
        "sequential_one_execute_per_release_rate": seq_rate,
        "speedup_vs_sequential": value / seq_rate,
        "particle_steps_per_run": total / args.steps,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def precision_workload(args, rank, world, local):
    """2-D surface field on a 1/12 degree grid (4320 x 2160), 60 daily snapshots,
    50M particles, RK4 dt 1 h for 60 days plus Brownian motion K = 10 m^2/s.
    Times the cell-index + FP32-offset form on FP16/BF16 storage and plain FP32
    on FP32 storage on the same workload; reports the speedup, the position
    error against the FP64 oracle on a 1e5-particle subset, and the diffusion
    variance against 2Kt."""
    import torch
    import ctypes as C
    import oracle as O
    import paper_1707_05163_gb300 as pg
    import synth
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    days = args.days if args.days != 30.0 else 60.0
    n = args.particles if args.particles != 10_000_000 else 50_000_000
    nt = 60
    gf = synth.GlobalField(res_deg=1.0 / 12.0, nz=1, nt=nt, seed=3, period=nt * DAY)
    kind = 0 if args.storage == "f16" else 1
    fs_q = pg.FieldSet(gf.lon, gf.lat, None, mesh="spherical", periodic_lon=True, nfields=2,
                       storage=args.storage)
    fs_32 = pg.FieldSet(gf.lon, gf.lat, None, mesh="spherical", periodic_lon=True, nfields=2,
                        storage="f32")
    for fs in (fs_q, fs_32):
        fs.set_times(gf.times, gf.period)
    host32 = np.empty((nt, 2, 1, gf.ny, gf.nx), dtype=np.float32)
    hostq = np.empty((nt, 2, 1, gf.ny, gf.nx), dtype=np.float32)
    for s in range(nt):
        slab = gf.base2d_torch(s, dev).to(torch.float32)[:, None]
        fs_q.load_snapshot(s, slab)
        fs_32.load_snapshot(s, slab)
        host32[s] = slab.cpu().numpy()
        for f in range(2):
            q, sc = O.quantise(host32[s, f], kind)
            assert sc == fs_q.scale(s, f)
            hostq[s, f] = O.dequantise(q, kind, sc).astype(np.float32)
        del slab
    lon, lat, _ = synth.uniform_particles(n, 3, (0.0, 360.0), (-80.0, 80.0), dtype=np.float32)
    dl, da = torch.from_numpy(lon).to(dev), torch.from_numpy(lat).to(dev)
    K = 10.0
    kern = pg.Kernel("rk4", ("brownian",), kh=K)
    runtime = days * DAY

    def run(fs, pos, timed):
        ps = pg.ParticleSet(fs, dl, da, pos=pos, seed=3)
        ps.set_tune(args.block, args.resort_steps, args.chunk_steps)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        steps = ps.execute(kern, runtime, 3600.0)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        return ps, steps, dt

    rates = {}
    finals = {}
    for name, fs, pos in (("cell_" + args.storage, fs_q, "cell"), ("plain_f32", fs_32, "f32")):
        for _ in range(args.warmup):
            ps, _, _ = run(fs, pos, False)
            ps.destroy()
        tot_s, tot_t = 0, 0.0
        for _ in range(args.steps):
            ps, st, dt = run(fs, pos, True)
            tot_s += st
            tot_t += dt
            sub = 100_000
            g = ps.get()
            finals[name] = {k: v[:sub] for k, v in g.items()}
            ps.destroy()
        rates[name] = tot_s / tot_t
    # oracle on the first 1e5 ids: on the dequantised field and on the FP32 field
    sub = min(100_000, n)
    cores = len(os.sched_getaffinity(0))
    errs = {}
    ospec = dict(lon=gf.lon, lat=gf.lat, depth=np.zeros(1), times=gf.times)

    # error against time: the state at these days (the last one the horizon)
    stops = [d for d in (1.0, 7.0, 30.0) if d < days] + [days]

    def oracle_final(data):
        """The oracle on the first `sub` particles; returns the state at each
        stop (the last one is the final state) and its particle-steps/s."""
        f = O.Field(gf.lon, gf.lat, np.zeros(1), gf.times, data, 1, True, gf.period)
        st = [np.array(lon[:sub], np.float64), np.array(lat[:sub], np.float64), np.zeros(sub),
              np.zeros(sub), np.arange(sub, dtype=np.uint64), np.zeros(sub, np.uint32),
              np.zeros(sub, np.uint8)]
        t0 = time.perf_counter()
        done = 0
        at = {}
        for d in stops:
            done += O.run(f, O.Kernel(O.RK4, O.BROWNIAN, K, 0.0, 3), *st, 3600.0, d * DAY, runtime,
                          nthreads=cores)
            at[d] = [a.copy() for a in st]
        return at, done / (time.perf_counter() - t0)

    def gpu_at_stops(fs, pos):
        """The same form run again with stops (launch boundaries do not change
        FP32 results); the first `sub` particles' state at each stop."""
        ps = pg.ParticleSet(fs, dl, da, pos=pos, seed=3)
        ps.set_tune(args.block, args.resort_steps, args.chunk_steps)
        out, t = {}, 0.0
        for d in stops:
            ps.execute(kern, d * DAY - t, 3600.0)
            t = d * DAY
            g = ps.get()
            out[d] = {k: v[:sub] for k, v in g.items()}
        ps.destroy()
        return out

    def err_cells(g, st):
        ok = (st[6] == 0) & (g["status"] == 0)
        dx = 1.0 / 12.0
        dlon = (g["lon"] - st[0] + 180.0) % 360.0 - 180.0
        e = np.maximum(np.abs(dlon), np.abs(g["lat"] - st[1])) / dx
        return {"mean": float(np.mean(e[ok])), "max": float(np.max(e[ok])),
                "status_equal": bool((st[6] == g["status"]).all())}

    at_q, orate = oracle_final(hostq)
    at_32, _ = oracle_final(host32)
    st_q, st_32 = at_q[days], at_32[days]
    qname = "cell_" + args.storage
    errs[qname + "_vs_oracle_same_field"] = err_cells(finals[qname], st_q)
    errs[qname + "_vs_oracle_fp32_field"] = err_cells(finals[qname], st_32)
    errs["plain_f32_vs_oracle_fp32_field"] = err_cells(finals["plain_f32"], st_32)
    gq, g32 = gpu_at_stops(fs_q, "cell"), gpu_at_stops(fs_32, "f32")
    errs_vs_time = {
        f"{d:g}_days": {
            qname + "_vs_oracle_same_field": err_cells(gq[d], at_q[d])["mean"],
            qname + "_vs_oracle_fp32_field": err_cells(gq[d], at_32[d])["mean"],
            "plain_f32_vs_oracle_fp32_field": err_cells(g32[d], at_32[d])["mean"]}
        for d in stops}
    # diffusion variance against 2 K t on a zero-velocity copy of the grid
    fz = pg.FieldSet(gf.lon, gf.lat, None, mesh="spherical", periodic_lon=True, nfields=2,
                     storage=args.storage)
    fz.set_times(np.zeros(1))
    fz.load_snapshot(0, np.zeros((2, 1, gf.ny, gf.nx), np.float32))
    nb = 1_000_000
    pz = pg.ParticleSet(fz, np.full(nb, 180.0), np.zeros(nb), pos="cell", seed=5)
    pz.execute(pg.Kernel("rk4", ("brownian",), kh=K), DAY, 3600.0)
    m = pz.moments()
    D = 1852.0 * 60.0
    var_lat = (m[5] / m[0] - (m[2] / m[0]) ** 2) * D * D
    var_lon = (m[4] / m[0] - (m[1] / m[0]) ** 2) * D * D
    line = {
        "metric": METRIC, "value": rates[qname], "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 offsets + " + args.storage,
        "data": "synthetic (seeded k^-3 random streamfunction field, uniform particles)",
        "config": {"workload": f"2-D RK4 + Brownian K=10, global 1/12 deg 4320x2160, {nt} daily "
                               f"snapshots ({args.storage} + per-snapshot FP32 scale), {n} "
                               f"particles, dt 1 h, {days:g} days", "form": "cell index + FP32 offset"},
        "plain_fp32_rate": rates["plain_f32"], "speedup_vs_plain_fp32": rates[qname] / rates["plain_f32"],
        "error_cells": errs,
        "mean_error_cells_vs_time": errs_vs_time,
        "diffusion_variance_over_2Kt_1day": {"lat": var_lat / (2 * K * DAY),
                                             "lon_at_equator": var_lon / (2 * K * DAY), "n": nb},
        "cpu_baseline": {"value": orate, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"first {sub} particles, full {days:g}-day horizon"},
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
