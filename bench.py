"""Benchmark: implicit backward-Euler steps per second of the surface-energy APIC-MPM
path on one GB300, plus the Hessian-vector operator's roofline.

Workload (default ``incline``): 256^3 grid, dx = 1/256, 40 droplets above a
30-degree slip plane, radii uniform in [9.3, 24.8] cells (about 8M interior
particles at 8 per cell, ~0.3M surface samples), gravity -9.8, interface
dependent surface coefficients (liquid-gas 1.0, effective solid-liquid 0.5 for a
120-degree contact angle), dt = 1e-3, Newton tolerance 1e-6 with CG. Seeded
synthetic input (no dataset exists for this path).

A step is one full pass of the method: resample (sort, closest parent, balance
particles, split) + P2G + heat solve (thermal scenes) + Newton-CG + G2P/merge.

Reported (one JSON line on rank 0):
  value        implicit steps/s, float32 operator + float64 reductions, inputs
               resident in HBM; the state (~2 GB) exceeds L2 between steps
  roofline     the Hessian-vector kernel: algorithmic bytes per launch / its mean
               CUDA-event duration inside the timed steps, against measured HBM
  e2e          the same steps/s through the C ABI with host buffers: particle and
               surface state copied in from pinned host memory and back out into
               it every step
  fp64_form    the all-float64 GPU form on the same workload (fewer steps)
  cpu_baseline the FP64 numpy oracle on a bounded sample of the workload (a
               16^3-cell window at the lower surface of its smallest droplet,
               or around the centroid of a scene without droplets; same dx,
               parameters and plane), scaled per particle to the full
               workload; one host thread (BLAS pools pinned to 1)
  --impl reference: the oracle alone, timed on the host, same metric.
Multi-GPU (torchrun): replicas only -- every rank advances its own copy of the
workload; value is the sum over ranks (weak scaling, no collective on the path).
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

# the oracle baseline runs on one host thread: pin the BLAS pools before numpy loads
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2101_12408_gb300 import scenes  # noqa: E402

METRIC = "implicit steps/sec (float32 operator + float64 reductions)"
UNIT = "steps/s"
# ncu DRAM traffic (read + write bytes) of one Hessian-operator apply at the
# full workload, from the 20-droplet capture in
# profiles/apply_cg_kernels_incline20_fp32.md scaled by the units processed:
# k_apply_cell (188.6 MB, particles and samples) x 8272476 / 5128948 particles
# plus k_apply_general (0.07 MB) x 317603 / 185006 samples. k_apply_cell's code
# is unchanged since that capture. k_apply_general has changed since (its
# particle loop and the projected solid maps), but this workload gives it no
# particles: its share is the scan of an empty list.
NCU_TRAFFIC_BYTES = 304312853


def make_workload(name, drops=40):
    if name == "incline":
        return scenes.incline(n_drops=drops)
    if name == "film":
        return scenes.film()
    if name == "droplet":
        return scenes.droplet()
    if name == "wax":
        return scenes.wax()
    raise ValueError(name)


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        v = pk.get("hbm_gbs")
        if v:
            return float(v), "measured"
    except (OSError, ValueError):
        pass
    return 6800.0, "fallback"


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def algorithmic_bytes(ctx, sc, rsize):
    """Bytes one Hessian-operator launch (projected form, as CG applies it) must
    move: the packed record of a liquid particle (position in its block and
    kappa, 4 values); a solid particle (position in its block and the iterate's
    symmetric 9x9 projected-Hessian map, 3 + 45 values); a surface sample (position in its block and
    the iterate's symmetric 9x9 Hessian map, 3 + 45 values); an active node (the
    direction read and the product written, 3 components each)."""
    p = ctx.get_particles(0)
    nsol = int(np.sum(p["phase"] == 1))
    nliq = ctx.np[0] - nsol
    m = ctx.get_grid(0, 0)
    g_active = int(np.sum(m > 0))
    b = rsize * (nliq * 4 + nsol * (3 + 45) + ctx.ns[0] * (3 + 45) + g_active * 6)
    return b, dict(liquid=nliq, solid=nsol, surface=ctx.ns[0], active_nodes=g_active)


def run_oracle_sample(sc, steps):
    """FP64 oracle on the workload's window sample; returns seconds per step and the sample."""
    import oracle
    from scipy.spatial import cKDTree  # noqa: F401  (scipy present on both machines)
    sample = sample_scene(sc)
    sim = oracle.OracleSim(sample)
    times = []
    for _ in range(steps):
        t = time.perf_counter()
        sim.step()
        times.append(time.perf_counter() - t)
    return times, sample


SAMPLE_CELLS = 16


def sample_where(sc):
    """Where `sample_scene` puts its window, in words."""
    if "radii" in sc.meta:
        return "at the lower surface of the smallest droplet"
    return "around the particles' centroid"


def sample_scene(sc, size=SAMPLE_CELLS):
    """A bounded piece of the workload for the CPU oracle: the particles and
    surface samples in a `size`^3-cell window (same dx, parameters and plane)
    around the lower surface of the smallest droplet, or around the particles'
    centroid in a scene without droplets."""
    if "radii" in sc.meta:
        k = int(np.argmin(sc.meta["radii"]))
        c = sc.meta["centers"][k] - np.array([0.0, sc.meta["radii"][k] - 3 * sc.dx, 0.0])
        return scenes.window(sc, c, size, name=f"incline_window{size}")
    c = sc.x.mean(0)
    return scenes.window(sc, c, size, name=f"{sc.name}_window{size}")


def job_rate(units, elapsed_ms, device=None):
    """Whole-job throughput of replicas: the units all ranks processed divided by
    the slowest rank's time. Returns (units / s, the slowest time in ms). Without an
    initialised process group it is the local rate."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return units / (elapsed_ms * 1e-3), elapsed_ms
    t = torch.tensor([float(elapsed_ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    tdist.all_reduce(u, op=tdist.ReduceOp.SUM)
    return float(u.item()) / (float(t.item()) * 1e-3), float(t.item())


def bench_ours(args, rank, world):
    import torch
    from paper_2101_12408_gb300 import mpm

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    sc = make_workload(args.workload, args.drops)
    stream = torch.cuda.current_stream()
    prec = mpm.PREC_FP32_FP64RED if args.precision == "fp32" else mpm.PREC_FP64
    ctx = mpm.Context(sc, precision=prec, stream=stream.cuda_stream, max_blocks=args.max_blocks,
                      surface_capacity_factor=2.0)
    ctx.load_scene(0)
    for _ in range(args.warmup):
        ctx.step()
    dist = world > 1
    if dist:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index)
    clocks.start()
    ctx.profile_enable(True)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    stats = []
    for _ in range(args.steps):
        stats.append(ctx.step()[0])
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        torch.distributed.barrier()
    elapsed_ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    prof = ctx.profile()
    ctx.profile_enable(False)
    steps_per_s, elapsed_ms = job_rate(args.steps, elapsed_ms, dev)
    rsize = 4 if prec == mpm.PREC_FP32_FP64RED else 8
    abytes, counts = algorithmic_bytes(ctx, sc, rsize)
    apply_avg_ms = prof["apply_ms"] / max(prof["apply_launches"], 1)
    peak, peak_kind = measured_peak()
    achieved = abytes / (apply_avg_ms * 1e-3) / 1e9
    out = {
        "steps_per_s": steps_per_s,
        "ms_per_step": elapsed_ms / args.steps,
        "prof": prof,
        "stats": stats,
        "clocks": clk,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": NCU_TRAFFIC_BYTES, "peak_source": peak_kind, "kernel": "k_apply (Hessian-vector)",
                     "bytes_per_launch": abytes, "launch_ms": apply_avg_ms,
                     "launches": prof["apply_launches"]},
        "counts": dict(counts, **{"grid_blocks": ctx.counts()["blocks"], "work_blocks": ctx.counts()["work_blocks"]}),
        "applies_per_s": prof["apply_launches"] / (elapsed_ms * 1e-3),
    }
    # end to end through host buffers: state in from host memory, step, state back out
    if args.e2e_steps > 0:
        tdt = {np.dtype(np.float64): torch.float64, np.dtype(np.uint8): torch.uint8, np.dtype(np.int32): torch.int32}

        def pinned(a):
            # a page-locked host copy: the step's inputs and outputs live in pinned memory
            buf = torch.empty(a.shape, dtype=tdt[a.dtype], pin_memory=True).numpy()
            buf[...] = a
            return buf

        cur = sc.copy()
        p = ctx.get_particles(0)
        srf = ctx.get_surface(0)
        pf = ("x", "v", "A", "J", "F", "T", "gradT", "phase")
        for f in pf:
            setattr(cur, f, pinned(p[f]))
        for f in ("m", "V0", "b", "Tbar"):
            setattr(cur, f, pinned(np.ascontiguousarray(getattr(sc, f))))
        cur.s, cur.dA, cur.kind = pinned(srf["s"]), pinned(srf["dA"]), pinned(srf["kind"])
        # each step's outputs land in the arrays the next step loads
        pout = {f: getattr(cur, f) for f in pf}
        sout = dict(s=cur.s, dA=cur.dA, kind=cur.kind, gamma=pinned(srf["gamma"]), parent=pinned(srf["parent"]),
                    b=pinned(srf["b"]))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            ctx.load_scene(0, cur)
            ctx.step()
            ctx.get_particles(0, out=pout)
            ctx.get_surface(0, out=sout)
        torch.cuda.synchronize()
        e2e_rate, _ = job_rate(args.e2e_steps, (time.perf_counter() - t0) * 1e3, dev)
        n, ns = ctx.np[0], ctx.ns[0]
        h2d = n * (3 + 3 + 9 + 1 + 1 + 1 + 9 + 1 + 3) * 8 + n + ns * (3 + 3 + 1 + 1) * 8 + ns
        d2h = n * (3 + 3 + 9 + 1 + 9 + 1 + 3) * 8 + n + ns * (3 + 3 + 1 + 3) * 8 + ns + ns * 4
        out["e2e"] = {"value": e2e_rate, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                      "d2h_bytes_per_step": int(d2h)}
    # surface regeneration (mpm_generate_surface), timed once on the final state,
    # outside the timed steps (the timed steps carry their samples)
    if args.surface_gen:
        ctx.generate_surface(1)   # warm-up (grows the triangle buffer)
        torch.cuda.synchronize()
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        cnt = ctx.generate_surface(2)
        g1.record(stream)
        torch.cuda.synchronize()
        out["surface_generation"] = {"ms": g0.elapsed_time(g1), "samples": int(cnt[0]),
                                     "carried_samples": int(sc.n_surface)}
    ctx.close()
    # all-float64 form on the same workload
    if args.fp64_steps > 0 and prec == mpm.PREC_FP32_FP64RED:
        ctx = mpm.Context(sc, precision=mpm.PREC_FP64, stream=stream.cuda_stream, max_blocks=args.max_blocks)
        ctx.load_scene(0)
        ctx.step()
        ctx.profile_enable(True)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st64 = [ctx.step()[0] for _ in range(args.fp64_steps)]
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        p64 = ctx.profile()
        out["fp64_form"] = {"steps_per_s": args.fp64_steps / (ms * 1e-3), "ms_per_step": ms / args.fp64_steps,
                            "apply_launch_ms": p64["apply_ms"] / max(p64["apply_launches"], 1),
                            "newton_iters": [s["newton_iters"] for s in st64],
                            "cg_iters": [s["cg_iters"] for s in st64],
                            "residual_rel": [s["residual"] / max(s["residual0"], 1e-300) for s in st64]}
        ctx.close()
    return out, sc


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="incline")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--cpu-steps", type=int, default=2)
    ap.add_argument("--surface-gen", type=int, default=1, help="time one surface regeneration (0: skip)")
    ap.add_argument("--drops", type=int, default=40, help="droplets in the incline workload")
    ap.add_argument("--max-blocks", type=int, default=0, help="grid block capacity (0: whole grid)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))

    if args.impl == "reference":
        if rank != 0:
            return
        sc = make_workload(args.workload, args.drops)
        times, sample = run_oracle_sample(sc, args.warmup + args.steps)
        t = float(np.mean(times[args.warmup:])) if args.steps > 0 else float("nan")
        scale = sample.n_particles / sc.n_particles
        val = scale / t
        line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / val, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": args.workload, "particles": sc.n_particles},
                "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                                 "sample": f"{sample.n[0]}^3-cell window {sample_where(sc)} "
                                           f"({sample.n_particles} of {sc.n_particles} particles, "
                                           f"{sample.n_surface} samples) per step, seconds per step scaled by "
                                           f"particle count ({scale:.5f})"},
                "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    res, sc = bench_ours(args, rank, world)
    if rank != 0:
        return
    cpu = None
    if args.cpu_steps > 0:
        times, sample = run_oracle_sample(sc, args.cpu_steps)
        t = float(np.mean(times))
        scale = sample.n_particles / sc.n_particles
        cpu = {"value": scale / t, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{sample.n[0]}^3-cell window {sample_where(sc)} "
                         f"({sample.n_particles} of {sc.n_particles} particles, {sample.n_surface} samples, "
                         f"{args.cpu_steps} steps), seconds per step scaled by particle count"}
    prof = res["prof"]
    line = {
        "metric": METRIC, "value": res["steps_per_s"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "grid": list(sc.n), "dx": sc.dx, "particles": sc.n_particles,
                   "surface_samples": sc.n_surface, "dt": sc.params.dt, "newton_tol": sc.params.newton_tol,
                   "l2": "inputs larger than L2 (particle state ~2 GB)", "parallelism": "replicas"},
        "roofline": res["roofline"],
        "cpu_baseline": cpu,
        "e2e": res.get("e2e"),
        "gpu_launches": prof["kernel_launches"],
        "clocks": res["clocks"],
        "hessian_applies_per_s": res["applies_per_s"],
        "fp64_form": res.get("fp64_form"),
        "phases_ms_per_step": {k: v / args.steps for k, v in prof["phase_ms"].items()},
        "surface_generation": res.get("surface_generation"),
        "cg_launch": {"ctas_per_sm": prof["cg_ctas_per_sm"], "iters_per_check": prof["cg_chunk"],
                      "cuda_graphs": bool(prof["cg_graphs"]), "graph_error": prof["cg_graph_error"]},
        "newton_iters": [s["newton_iters"] for s in res["stats"]],
        "cg_iters": [s["cg_iters"] for s in res["stats"]],
        "residual_rel": [s["residual"] / max(s["residual0"], 1e-300) for s in res["stats"]],
        "counts": res["counts"],
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()
