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
  fp64_form    the all-float64 GPU form on the same workload, the same warm-up
               and the same number of timed steps from the same initial state
  hessian_apply  the operator alone: 200 back-to-back applications on the
               frozen Newton state after one more step, both forms
  regenerated_surface  steps/s with a new surface generated before every step
  cpu_baseline the FP64 numpy oracle on bounded samples of the workload (16^3-cell
               windows around the lower surfaces of its droplets, or around the
               centroid of a scene without droplets; same dx, parameters and
               plane), one window per host core in separate processes, scaled
               per particle to the full workload; the one-thread figure beside it,
               and one step of the whole 32^3 droplet on one thread (a complete
               workload, no scaling)
  operator_tile  the record rows per bulk copy the autotuner picked for the
               Hessian operator
  --impl reference: the oracle alone, timed the same way on the host cores.
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
# full workload, with the SHA-256 of the operator's source files it was
# measured on. When those files have changed since, the line reports no traffic.
# Captured on the 20-droplet variant of the inclined-plane workload (three
# launches, 188.2 MB each against 137.9 MB of algorithmic bytes) and scaled to
# the full 8.27M-particle launch by its algorithmic bytes.
NCU_TRAFFIC = {"bytes_per_apply": 309628932,
               "source_sha256": "7890972c97652ef596a52a3114b444117caaff1e765b4b86414c6e6662cf9f9a"}
OPERATOR_SOURCES = ("paper_2101_12408_gb300/csrc/newton.cu", "paper_2101_12408_gb300/csrc/common.cuh")
# the parts of newton.cu the operator's launch runs: the record packing and the
# operator section (argument struct, transforms, kernels, launch helper)
OPERATOR_REGIONS = (("__global__ void k_pack_volume(", "__global__ void k_pack_surface("),
                    ("// Hessian-vector operator (the hot kernel)", "// Per-iterate projected Hessian of each solid particle"))


def operator_source_hash():
    import hashlib
    h = hashlib.sha256()
    with open(os.path.join(ROOT, OPERATOR_SOURCES[0])) as fh:
        text = fh.read()
    for a, b in OPERATOR_REGIONS:
        i = text.index(a)
        h.update(text[i:text.index(b, i)].encode())
    with open(os.path.join(ROOT, OPERATOR_SOURCES[1]), "rb") as fh:
        h.update(fh.read())
    return h.hexdigest()


def measured_traffic(workload, drops):
    """The captured traffic, for the workload it was scaled to (the 40-droplet
    inclined plane) and the operator source it was captured on; else None."""
    if workload != "incline" or drops != 40:
        return None
    if NCU_TRAFFIC["bytes_per_apply"] is None or NCU_TRAFFIC["source_sha256"] != operator_source_hash():
        return None
    return NCU_TRAFFIC["bytes_per_apply"]


def make_workload(name, drops=40):
    if name == "incline":
        return scenes.incline(n_drops=drops)
    if name == "film":
        return scenes.film()
    if name == "film27":
        # the film at the configuration's particle count: 27 particles per cell
        # (a 3x3x3 sub-cell lattice) in the same 6-cell layer, 2.49M particles
        return scenes.film(ppc_axis=3)
    if name == "droplet":
        return scenes.droplet()
    if name == "wax":
        return scenes.wax()
    if name == "batch":
        return scenes.batch()
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


def algorithmic_bytes(ctx, rsize):
    """Bytes one Hessian-operator launch (projected form, as CG applies it) must
    move, over every scene of the context: the packed record of a liquid particle
    (position in its block and kappa, 4 values); a solid particle (position in its
    block and the iterate's symmetric 9x9 projected-Hessian map, 3 + 45 values); a
    surface sample (position in its block and the iterate's symmetric 9x9 Hessian
    map, 3 + 45 values); an active node (the direction read and the product
    written, 3 components each)."""
    nliq = nsol = nsurf = g_active = 0
    for k in range(len(ctx.scenes)):
        p = ctx.get_particles(k)
        ns_ = int(np.sum(p["phase"] == 1))
        nsol += ns_
        nliq += ctx.np[k] - ns_
        nsurf += ctx.ns[k]
        g_active += int(np.sum(ctx.get_grid(k, 0) > 0))
    b = rsize * (nliq * 4 + nsol * (3 + 45) + nsurf * (3 + 45) + g_active * 6)
    return b, dict(liquid=nliq, solid=nsol, surface=nsurf, active_nodes=g_active)


SAMPLE_CELLS = 16


def _scenes_of(sc):
    return sc if isinstance(sc, list) else [sc]


def total_particles(sc):
    return sum(s.n_particles for s in _scenes_of(sc))


def sample_where(sc):
    """Where `sample_windows` puts its windows, in words."""
    s0 = _scenes_of(sc)[0]
    if "radii" in s0.meta:
        return "at the lower surfaces of its droplets, smallest first"
    return "around the particles' centroids"


def sample_windows(sc, count, size=SAMPLE_CELLS):
    """Bounded pieces of the workload for the CPU oracle: the particles and surface
    samples in `size`^3-cell windows (same dx, parameters and plane), one around
    the lower surface of each droplet (smallest first), or around the centroid of
    each scene of a workload without droplets."""
    out = []
    for s in _scenes_of(sc):
        if "radii" in s.meta:
            for k in np.argsort(s.meta["radii"]):
                c = s.meta["centers"][k] - np.array([0.0, s.meta["radii"][k] - 3 * s.dx, 0.0])
                out.append(scenes.window(s, c, size, name=f"{s.name}_window{size}_{k}"))
                if len(out) == count:
                    return out
        else:
            out.append(scenes.window(s, s.x.mean(0), size, name=f"{s.name}_window{size}"))
            if len(out) == count:
                return out
    while len(out) < count:   # fewer windows than cores: repeat them
        out.append(out[len(out) % max(1, len(out))])
    return out


def _oracle_worker(job):
    """One host process: the FP64 oracle on one window; seconds of each step."""
    sample, steps = job
    import oracle
    sim = oracle.OracleSim(sample)
    times = []
    for _ in range(steps):
        t = time.perf_counter()
        sim.step()
        times.append(time.perf_counter() - t)
    return sample.n_particles, times


def run_oracle(sc, steps, warmup, processes):
    """The oracle as it stands on `processes` host cores at once, each process on
    its own window (spawned processes, BLAS pools pinned to one thread each).
    Returns (full-workload steps/s, per-process particle counts, mean step seconds)."""
    import multiprocessing as mp
    wins = sample_windows(sc, processes)
    if processes == 1:
        res = [_oracle_worker((wins[0], warmup + steps))]
    else:
        with mp.get_context("spawn").Pool(processes) as pool:
            res = pool.map(_oracle_worker, [(w, warmup + steps) for w in wins])
    counts = [n for n, _ in res]
    secs = [float(np.mean(ts[warmup:])) if steps > 0 else float("nan") for _, ts in res]
    # the processes run side by side: their particle rates add up
    rate = sum(n / s for n, s in zip(counts, secs))
    return rate / total_particles(sc), counts, secs


def oracle_baseline(sc, steps, warmup=0, one_core_steps=None):
    """cpu_baseline object: every host core, with the one-core figure beside it
    (timed over `one_core_steps` steps without warm-up when given)."""
    cores = os.cpu_count() or 1
    if one_core_steps is None:
        v1, c1, s1 = run_oracle(sc, steps, warmup, 1)
    else:
        v1, c1, s1 = run_oracle(sc, one_core_steps, 0, 1)
    vn, cn, sn = run_oracle(sc, steps, warmup, cores) if cores > 1 else (v1, c1, s1)
    return {"value": vn, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} host processes side by side, each the FP64 oracle on its own {SAMPLE_CELLS}^3-cell "
                      f"window {sample_where(sc)} ({min(cn)}-{max(cn)} particles each, {steps} timed steps after "
                      f"{warmup}); particle rates summed and scaled to the {total_particles(sc)}-particle workload",
            "host_cpu_count": cores,
            "one_core": {"value": v1, "cores": 1, "particles": c1[0], "sec_per_step": s1[0]},
            "droplet_full": oracle_droplet_full()}


def oracle_droplet_full():
    """The oracle on the whole small droplet (32^3 grid, r = 8 cells, ~17k
    particles), one step on one core: a complete workload rather than a window."""
    import oracle
    sc = scenes.config(0)
    sim = oracle.OracleSim(sc)
    t = time.perf_counter()
    sim.step()
    sec = time.perf_counter() - t
    return {"particles": sc.n_particles, "surface_samples": sc.n_surface, "sec_per_step": sec,
            "steps_per_s": 1.0 / sec, "cores": 1}


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


def _timed_steps(ctx, stream, steps):
    import torch
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    stats = [ctx.step() for _ in range(steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1), stats


def _isolated_apply(ctx, n_applies):
    """One more step's resample, P2G and Newton solve, then the operator alone on
    that frozen state; the step is finished with G2P."""
    ctx.resample()
    ctx.p2g()
    ctx.newton_step()
    ms = ctx.profile_apply(n_applies)
    ctx.g2p()
    return ms


def bench_ours(args, rank, world):
    import torch
    from paper_2101_12408_gb300 import mpm

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    sc = make_workload(args.workload, args.drops)
    scl = _scenes_of(sc)
    stream = torch.cuda.current_stream()
    prec = mpm.PREC_FP32_FP64RED if args.precision == "fp32" else mpm.PREC_FP64
    ctx = mpm.Context(scl, precision=prec, stream=stream.cuda_stream, max_blocks=args.max_blocks,
                      surface_capacity_factor=2.0)
    for k in range(len(scl)):
        ctx.load_scene(k)
    for _ in range(args.warmup):
        ctx.step()
    dist = world > 1
    if dist:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index)
    clocks.start()
    ctx.profile_enable(True)
    elapsed_ms, stats = _timed_steps(ctx, stream, args.steps)
    if dist:
        torch.distributed.barrier()
    clk = clocks.stop()
    prof = ctx.profile()
    ctx.profile_enable(False)
    steps_per_s, elapsed_ms = job_rate(args.steps, elapsed_ms, dev)
    rsize = 4 if prec == mpm.PREC_FP32_FP64RED else 8
    abytes, counts = algorithmic_bytes(ctx, rsize)
    apply_avg_ms = prof["apply_ms"] / max(prof["apply_launches"], 1)
    peak, peak_kind = measured_peak()
    achieved = abytes / (apply_avg_ms * 1e-3) / 1e9
    cnt = ctx.counts()
    out = {
        "steps_per_s": steps_per_s,
        "ms_per_step": elapsed_ms / args.steps,
        "prof": prof,
        "stats": stats,
        "clocks": clk,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": measured_traffic(args.workload, args.drops), "peak_source": peak_kind,
                     "kernel": "k_apply_pair + k_apply_surf + k_apply_general (Hessian-vector operator)",
                     "bytes_per_launch": abytes, "launch_ms": apply_avg_ms, "launches": prof["apply_launches"]},
        "counts": dict(counts, grid_blocks=cnt["blocks"], work_blocks=cnt["work_blocks"]),
        "applies_per_s": prof["apply_launches"] / (elapsed_ms * 1e-3),
    }
    # the operator alone on a frozen Newton state
    iso = {}
    if args.apply_bench > 0:
        ms = _isolated_apply(ctx, args.apply_bench)
        iso["fp32" if rsize == 4 else "fp64"] = {
            "ms_per_apply": ms, "applies_per_s": 1e3 / ms, "gbs": abytes / (ms * 1e-3) / 1e9,
            "frac": abytes / (ms * 1e-3) / 1e9 / peak, "bytes_per_apply": abytes, "applies": args.apply_bench}
    # end to end through host buffers: state in from host memory, step, state back out
    if args.e2e_steps > 0:
        tdt = {np.dtype(np.float64): torch.float64, np.dtype(np.uint8): torch.uint8, np.dtype(np.int32): torch.int32}

        def pinned(a):
            # a page-locked host copy: the step's inputs and outputs live in pinned memory
            buf = torch.empty(a.shape, dtype=tdt[a.dtype], pin_memory=True).numpy()
            buf[...] = a
            return buf

        pf = ("x", "v", "A", "J", "F", "T", "gradT", "phase")
        curs, pouts, souts = [], [], []
        for k, s0 in enumerate(scl):
            cur = s0.copy()
            p = ctx.get_particles(k)
            srf = ctx.get_surface(k)
            for f in pf:
                setattr(cur, f, pinned(p[f]))
            for f in ("m", "V0", "b", "Tbar"):
                setattr(cur, f, pinned(np.ascontiguousarray(getattr(s0, f))))
            cur.s, cur.dA, cur.kind = pinned(srf["s"]), pinned(srf["dA"]), pinned(srf["kind"])
            curs.append(cur)
            # each step's outputs land in the arrays the next step loads
            pouts.append({f: getattr(cur, f) for f in pf})
            souts.append(dict(s=cur.s, dA=cur.dA, kind=cur.kind, gamma=pinned(srf["gamma"]),
                              parent=pinned(srf["parent"]), b=pinned(srf["b"])))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            for k in range(len(scl)):
                ctx.load_scene(k, curs[k])
            ctx.step()
            for k in range(len(scl)):
                ctx.get_particles(k, out=pouts[k])
                ctx.get_surface(k, out=souts[k])
        torch.cuda.synchronize()
        e2e_rate, _ = job_rate(args.e2e_steps, (time.perf_counter() - t0) * 1e3, dev)
        n, ns = sum(ctx.np), sum(ctx.ns)
        h2d = n * (3 + 3 + 9 + 1 + 1 + 1 + 9 + 1 + 3) * 8 + n + ns * (3 + 3 + 1 + 1) * 8 + ns
        d2h = n * (3 + 3 + 9 + 1 + 9 + 1 + 3) * 8 + n + ns * (3 + 3 + 1 + 3) * 8 + ns + ns * 4
        out["e2e"] = {"value": e2e_rate, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                      "d2h_bytes_per_step": int(d2h)}
    # surface regeneration (mpm_generate_surface): once on its own, then steps
    # that regenerate the surface before every step (section "Discretization",
    # step 1); the headline steps carry their samples
    if args.surface_gen:
        ctx.generate_surface(1)   # warm-up (grows the triangle buffer)
        torch.cuda.synchronize()
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        cnt_g = ctx.generate_surface(2)
        g1.record(stream)
        torch.cuda.synchronize()
        out["surface_generation"] = {"ms": g0.elapsed_time(g1), "samples": int(np.sum(cnt_g)),
                                     "carried_samples": int(sum(s0.n_surface for s0 in scl))}
    if args.regen_steps > 0:
        ctx.step()   # warm-up on the regenerated surface
        torch.cuda.synchronize()
        r0 = torch.cuda.Event(enable_timing=True)
        r1 = torch.cuda.Event(enable_timing=True)
        r0.record(stream)
        rst = []
        for k in range(args.regen_steps):
            ctx.generate_surface(100 + k)
            rst.append(ctx.step())
        r1.record(stream)
        torch.cuda.synchronize()
        ms = r0.elapsed_time(r1)
        out["regenerated_surface"] = {"steps_per_s": args.regen_steps / (ms * 1e-3),
                                      "ms_per_step": ms / args.regen_steps, "steps": args.regen_steps,
                                      "surface_samples": int(sum(ctx.ns)),
                                      "newton_iters": [s[0]["newton_iters"] for s in rst],
                                      "cg_iters": [s[0]["cg_iters"] for s in rst],
                                      "residual_rel": [s[0]["residual"] / max(s[0]["residual0"], 1e-300)
                                                       for s in rst]}
    ctx.close()
    # all-float64 form: same workload, warm-up and timed step count, from the same
    # initial state
    if args.fp64_steps != 0 and prec == mpm.PREC_FP32_FP64RED:
        n64 = args.steps if args.fp64_steps < 0 else args.fp64_steps
        w64 = args.warmup if args.fp64_steps < 0 else 1
        ctx = mpm.Context(scl, precision=mpm.PREC_FP64, stream=stream.cuda_stream, max_blocks=args.max_blocks,
                          surface_capacity_factor=2.0)
        for k in range(len(scl)):
            ctx.load_scene(k)
        for _ in range(w64):
            ctx.step()
        torch.cuda.synchronize()
        ctx.profile_enable(True)
        ms, st64 = _timed_steps(ctx, stream, n64)
        p64 = ctx.profile()
        ctx.profile_enable(False)
        out["fp64_form"] = {"steps_per_s": n64 / (ms * 1e-3), "ms_per_step": ms / n64, "steps": n64,
                            "warmup": w64, "apply_launch_ms": p64["apply_ms"] / max(p64["apply_launches"], 1),
                            "newton_iters": [s[0]["newton_iters"] for s in st64],
                            "cg_iters": [s[0]["cg_iters"] for s in st64],
                            "residual_rel": [s[0]["residual"] / max(s[0]["residual0"], 1e-300) for s in st64]}
        if args.apply_bench > 0:
            ms = _isolated_apply(ctx, args.apply_bench)
            b64, _ = algorithmic_bytes(ctx, 8)
            iso["fp64"] = {"ms_per_apply": ms, "applies_per_s": 1e3 / ms, "gbs": b64 / (ms * 1e-3) / 1e9,
                           "frac": b64 / (ms * 1e-3) / 1e9 / peak, "bytes_per_apply": b64,
                           "applies": args.apply_bench}
        ctx.close()
    if iso:
        out["hessian_apply"] = iso
    return out, sc


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="incline", choices=["incline", "film", "film27", "droplet", "wax", "batch"])
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--fp64-steps", type=int, default=-1,
                    help="timed steps of the all-float64 form (-1: as many as --steps, after as many warm-up steps; "
                         "0: skip)")
    ap.add_argument("--apply-bench", type=int, default=200, help="isolated operator applications (0: skip)")
    ap.add_argument("--cpu-steps", type=int, default=1)
    ap.add_argument("--surface-gen", type=int, default=1, help="time one surface regeneration (0: skip)")
    ap.add_argument("--regen-steps", type=int, default=3, help="steps with a regenerated surface (0: skip)")
    ap.add_argument("--drops", type=int, default=40, help="droplets in the incline workload")
    ap.add_argument("--max-blocks", type=int, default=0, help="grid block capacity (0: whole grid)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))

    if args.impl == "reference":
        if rank != 0:
            return
        sc = make_workload(args.workload, args.drops)
        # the one-core figure beside the all-core one over two steps, so that the
        # whole run stays within a few minutes
        cpu = oracle_baseline(sc, args.steps, args.warmup, one_core_steps=min(args.steps, 2))
        val = cpu["value"]
        line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / val, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": args.workload, "particles": total_particles(sc)},
                "cpu_baseline": cpu,
                "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    res, sc = bench_ours(args, rank, world)
    if rank != 0:
        return
    cpu = oracle_baseline(sc, args.cpu_steps) if args.cpu_steps > 0 else None
    prof = res["prof"]
    scl = _scenes_of(sc)
    s0 = scl[0]
    cfg = {"workload": args.workload, "scenes": len(scl), "particles": total_particles(sc),
           "surface_samples": int(sum(s.n_surface for s in scl)), "dt": s0.params.dt,
           "newton_tol": s0.params.newton_tol, "l2": "inputs larger than L2 (particle state ~2 GB)",
           "parallelism": "replicas"}
    if len(scl) == 1:
        cfg.update(grid=list(s0.n), dx=s0.dx)
    else:
        cfg.update(grids=[list(s.n) for s in scl], particles_per_scene=[s.n_particles for s in scl])
    line = {
        "metric": METRIC, "value": res["steps_per_s"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64",
        "data": "synthetic",
        "config": cfg,
        "roofline": res["roofline"],
        "cpu_baseline": cpu,
        "e2e": res.get("e2e"),
        "gpu_launches": prof["kernel_launches"],
        "clocks": res["clocks"],
        "hessian_applies_per_s": res["applies_per_s"],
        "hessian_apply": res.get("hessian_apply"),
        "fp64_form": res.get("fp64_form"),
        "regenerated_surface": res.get("regenerated_surface"),
        "phases_ms_per_step": {k: v / args.steps for k, v in prof["phase_ms"].items()},
        "surface_generation": res.get("surface_generation"),
        "cg_launch": {"ctas_per_sm": prof["cg_ctas_per_sm"], "iters_per_check": prof["cg_chunk"],
                      "cuda_graphs": bool(prof["cg_graphs"]), "graph_error": prof["cg_graph_error"]},
        "operator_tile": {"record_rows_per_chunk": prof["op_rows_per_chunk"]},
        "newton_iters": [[s["newton_iters"] for s in st] for st in res["stats"]] if len(scl) > 1
        else [st[0]["newton_iters"] for st in res["stats"]],
        "cg_iters": [st[0]["cg_iters"] for st in res["stats"]] if len(scl) == 1
        else [max(s["cg_iters"] for s in st) for st in res["stats"]],
        "residual_rel": [max(s["residual"] / max(s["residual0"], 1e-300) for s in st) for st in res["stats"]],
        "counts": res["counts"],
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()
