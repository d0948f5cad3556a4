#!/usr/bin/env python
"""Benchmark of the fused two-component Shan-Chen D3Q19 evaporation step.

One benchmark step = one lattice time step of the workload.
Default workload: the 512^3 floating droplet (radius 96, centred; sinks at the
z-boundary planes z = 511 and z = 0; tau = 1, G = 3.6, rho_H = 0.03; seeded
+-1e-4 noise) with FP32 populations on one lattice updated in place (the AA
pattern), the large-droplet configuration of the precision study; its 20 GB of
populations exceed the 129 MB L2 many times, so no flush is needed between steps.
The same lattice is also timed with FP16 and BF16 offset storage
(`storage_variants`).

Metric: MLUPS (million site updates per second, both components per update).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload droplet_512|droplet_128|droplet_256|droplet_1024|film_4x4x128|ensemble_64|serve]
                    [--layout two|aa] [--storage f32|f16|bf16|f16s]

Under torchrun each rank advances its own copy of the lattice (independent
problems, no data exchange): weak scaling, value = all ranks' site updates /
the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_SITE = {"f32": 304, "f16": 152, "bf16": 152, "f16s": 152}  # read + write 2 x 19 populations
# bytes the in-place (AA) step moves per site: its Psi pass reads the 2 x 19
# populations and writes (Psi^r, Psi^b) in FP32, its collision reads them again
# with Psi and writes them back
AA_BYTES_PER_SITE = {k: 3 * v // 2 + 16 for k, v in BYTES_PER_SITE.items()}
PROFILE_DIR = os.path.join(ROOT, "profiles")
L2_BYTES = 129e6  # GB300 L2
# population layout of each workload unless --layout says otherwise: the droplets
# of 512^3 and more are the in-place (AA) configuration
DEFAULT_LAYOUT = {"droplet_256": "aa", "droplet_512": "aa", "droplet_1024": "aa"}
# the oracle's sample of a workload too large for it: the 128^3 droplet of the same
# recipe (radius / box = 0.1875), the crop-equivalent case of the precision study
ORACLE_CROP_EDGE = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="droplet_512")
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16", "f16s"])
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--zchunk", type=int, default=0)
    ap.add_argument("--layout", default=None, choices=["two", "aa", "slab"],
                    help="two population lattices, or one updated in place (half the memory), or one "
                         "lattice split along z over the ranks (two lattices per slab, ghost planes "
                         "exchanged every step); default: in place for the 256^3 - 1024^3 droplets, "
                         "two lattices otherwise")
    ap.add_argument("--staging", default="auto", choices=["auto", "thread", "rows", "persistent"],
                    help="how the step kernel gathers its populations (in place: persistent or the two-pass step)")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip timing the other storage types on the default workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="keep the automatic kernel configuration")
    ap.add_argument("--requests", type=int, default=40, help="serve workload: requests in the stream")
    ap.add_argument("--rate", type=float, default=20.0, help="serve workload: arrivals per second")
    ap.add_argument("--light-rate", type=float, default=4.0,
                    help="serve workload: arrivals per second of the lighter stream (a quarter as many requests)")
    args = ap.parse_args()
    if args.layout is None:
        args.layout = DEFAULT_LAYOUT.get(args.workload, "two")
    return args


def workload(name, storage, tile=0, zchunk=0, layout="two", staging="auto"):
    from paper_1701_03637_gb300.workloads import WORKLOADS
    params, init = WORKLOADS[name](storage=storage)
    params.update(tile=tile, zchunk=zchunk, layout=layout, staging=staging)
    return params, init


def describe(name, params, storage):
    n = params["nx"]
    geom = {0: "periodic", 1: f"planar sink z={params.get('sink_z0')} x{params.get('sink_layers')} layers",
            2: f"spherical sink R_H={params.get('R_H')}"}[params.get("geometry", 0)]
    shape = "film on a wall" if params.get("wall_thickness", 0) else "droplet"
    return (f"{name}: {params['nx']}x{params['ny']}x{params['nz']} two-component D3Q19 Shan-Chen {shape}, "
            f"{geom}, tau=1, G=3.6, rho_H={params['rho_H']}, {storage} populations, "
            + ("one lattice updated in place (AA pattern)" if params.get("layout") == "aa"
               else "two-lattice pull"))


ENSEMBLE_DESC = ("ensemble_64: 64 two-component D3Q19 Shan-Chen lattices, edges exp(U(ln 32, ln 96)) per axis, "
                 "even = planar film on a wall, odd = droplet, g ~ U(3.2, 3.8), tau ~ U(0.8, 1.2), master seed 3")


def serve_desc(args, storage):
    return (f"serve: {args.requests} requests, Poisson {args.rate}/s, cubic lattices edge exp(U(ln 32, ln 160)), "
            f"2000-20000 steps, films and droplets, g ~ U(3.2, 3.8), tau ~ U(0.8, 1.2), {storage} offsets, "
            f"master seed 4")


def source_digest():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1701_03637_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + b"\0" + fh.read())
    return h.hexdigest()[:16]


def profile_fields():
    """Machine-readable fields ("- key: `value`" lines) of every ncu summary under
    profiles/, one dict per file."""
    out = []
    try:
        names = sorted(os.listdir(PROFILE_DIR))
    except OSError:
        return out
    for name in names:
        if not name.endswith(".md"):
            continue
        kv = {"file": name}
        try:
            for ln in open(os.path.join(PROFILE_DIR, name)).read().splitlines():
                if ln.startswith("- ") and ":" in ln:
                    k, v = ln[2:].split(":", 1)
                    kv[k.strip()] = v.strip().strip("`")
        except OSError:
            continue
        out.append(kv)
    return out


def profiled_traffic(workload_name, storage, tile=None, zchunk=None, layout="two"):
    """DRAM bytes per time step of the dominant kernel from a committed ncu summary
    (dram_bytes_per_step, or dram_bytes_per_launch of a kernel that runs one step per
    launch), if one was taken on the current kernel source, this workload, storage,
    layout and launch configuration; None otherwise."""
    for kv in profile_fields():
        key = "dram_bytes_per_step" if "dram_bytes_per_step" in kv else "dram_bytes_per_launch"
        if key not in kv:
            continue
        if kv.get("source_digest") != source_digest() or kv.get("workload") != workload_name:
            continue
        if kv.get("storage") != storage or kv.get("layout", "two") != layout:
            continue
        if tile is not None and (kv.get("tile") != tile or kv.get("zchunk") != str(zchunk)):
            continue
        try:
            return float(kv[key])
        except ValueError:
            continue
    return None


def l2_note(pop_bytes):
    """How the timed steps relate to the L2: the populations the steps stream against
    its 129 MB."""
    if pop_bytes > L2_BYTES:
        return f"inputs larger than L2 (no flush): {pop_bytes / 1e9:.3g} GB of populations against 129 MB"
    return (f"populations fit in L2 ({pop_bytes / 1e6:.3g} MB < 129 MB): steps run back to back without a "
            f"flush, a warm-L2 figure")


def population_bytes(params, storage, layout):
    es = 4 if storage == "f32" else 2
    return params["nx"] * params["ny"] * params["nz"] * 38 * es * (1 if layout == "aa" else 2)


def arm_config(args, world):
    """The `config` of a line, the same for this library's arm and the oracle arm:
    it names the workload (sizes, storage, layout, how it meets the L2, how ranks
    share it) and nothing about kernels."""
    from paper_1701_03637_gb300.workloads import ensemble
    if args.workload == "ensemble_64":
        members = ensemble(64, 3, args.storage)
        sites = sum(p["nx"] * p["ny"] * p["nz"] for p, _ in members)
        return {"workload": ENSEMBLE_DESC, "sites": sites, "lattices": 64, "storage": args.storage,
                "layout": "two",
                "l2": l2_note(sum(population_bytes(p, args.storage, "two") for p, _ in members)),
                "parallelism": "one persistent launch per step over all members"
                               + (f"; members split over {world} ranks by size, no data exchange" if world > 1 else "")}
    if args.workload == "ncomp3_128":
        return {"workload": NCOMP_DESC, "sites": 128 ** 3, "components": 3, "storage": "f32", "layout": "two",
                "l2": l2_note(128 ** 3 * 3 * 19 * 4 * 2),
                "parallelism": f"independent replicas x{world}"}
    if args.workload == "serve":
        storage = args.storage if args.storage != "f32" else "f16"
        return {"workload": serve_desc(args, storage), "requests": args.requests, "rate_per_s": args.rate,
                "storage": storage, "layout": "two", "diag_every": 100,
                "l2": "resident lattices (up to the arena) stream through L2 each step; no flush",
                "parallelism": f"requests dispatched round-robin over {world} ranks, no data exchange"
                               if world > 1 else "one GPU"}
    params, _ = workload(args.workload, args.storage, args.tile, args.zchunk, args.layout)
    return workload_config(args, params, world)


def workload_config(args, params, world):
    """The `config` of both arms' lines: what the workload is, nothing about kernels."""
    return {"workload": describe(args.workload, params, args.storage),
            "sites": params["nx"] * params["ny"] * params["nz"], "lattices_per_gpu": 1,
            "storage": args.storage, "layout": args.layout,
            "l2": l2_note(population_bytes(params, args.storage, args.layout)),
            "parallelism": (f"one lattice split along z over {world} ranks, 2 ghost planes per side exchanged "
                            f"every step ({2 * 19 * 2 * params['nx'] * params['ny'] * (4 if args.storage == 'f32' else 2)}"
                            f" bytes per face)") if args.layout == "slab" else f"independent replicas x{world}"}


def launch_cfg(lat):
    info = lat.launch_info()
    return f"{info['tile_x']}x{info['tile_y']}", info["zchunk"]


def measured_peak_hbm():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples every 200 ms; keeps the rows taken inside [t0, t1]."""

    FIELDS = ("timestamp,index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        self.proc = None
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self, t0, t1, bus_id=None):
        rows = []
        try:
            for ln in open(self.path):
                parts = [p.strip() for p in ln.split(",")]
                if len(parts) < 11:
                    continue
                try:
                    ts = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                    ts += float("0." + parts[0].split(".")[1]) if "." in parts[0] else 0.0
                except Exception:
                    continue
                if bus_id and bus_id.lower() not in parts[2].lower():
                    continue
                if t0 - 0.25 <= ts <= t1 + 0.25:
                    rows.append(parts)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        mx = [float(r[4]) for r in rows if r[4].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[7 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(float(r[5]) for r in rows if r[5].replace(".", "").isdigit()) if rows else None}


def oracle_rate(params, init, budget_s, threads):
    """Time the FP64 oracle as it stands on the host cores: MLUPS over whole-lattice steps."""
    import oracle
    oracle.set_threads(threads)
    o = oracle.Lattice(params)
    o.init_shape(init)
    t = time.perf_counter()
    o.step(1)
    one = time.perf_counter() - t
    steps = max(1, int(budget_s / max(one, 1e-6)))
    t = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t
    n = params["nx"] * params["ny"] * params["nz"]
    return n * steps / dt / 1e6, steps


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def max_over_ranks(v, world, device="cpu"):
    """The largest of every rank's value (the slowest rank's time); world == 1
    needs no process group."""
    if world == 1:
        return float(v)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_results(res, world):
    """Every rank's served results, merged in request order (rank 0 reports them);
    world == 1 needs no process group."""
    if world == 1:
        return sorted(res, key=lambda r: r.rid)
    import torch.distributed as dist
    parts = [None] * world
    dist.all_gather_object(parts, list(res))
    return sorted((r for part in parts for r in part), key=lambda r: r.rid)


def sum_over_ranks(v, world, device="cpu"):
    """The sum of every rank's value; world == 1 needs no process group."""
    if world == 1:
        return float(v)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def replica_value(sites_per_rank, steps, world, ms_max):
    """Whole-job MLUPS of independent replicas: every rank's site updates over
    the slowest rank's time (weak scaling)."""
    return sites_per_rank * steps * world / (ms_max * 1e-3) / 1e6


def reference_lattices(args):
    """The lattices the oracle arm steps, each once per benchmark step: the workload's
    own lattice when it is small (the 4x4x128 film), a centred crop of a droplet
    workload sized to the time budget (same geometry and parameters, radius scaled),
    or, for the ensemble and the served stream, the workload's own lattices smallest
    first up to that size. Returns (lattices, sample description, workload label)."""
    from paper_1701_03637_gb300.workloads import WORKLOADS, droplet, ensemble, request_stream
    cores = host_cores()
    # calibrate on a 24^3 droplet, then size the sample so W + K steps take about 90 s
    p_probe, i_probe = droplet(24, 4.5, 1)
    rate, _ = oracle_rate(p_probe, i_probe, 0.5, cores)
    budget = max(512.0, rate * 1e6 * 90.0 / max(1, args.steps + args.warmup))
    name = args.workload
    if name in ("ensemble_64", "serve"):
        if name == "ensemble_64":
            pool = ensemble(64, 3, "f32")
        else:
            pool = [(p, i) for _, p, i, _ in request_stream(args.requests, args.rate, 4, storage="f32")]
        pool = sorted(pool, key=lambda m: m[0]["nx"] * m[0]["ny"] * m[0]["nz"])
        chosen, total = [], 0
        for p, i in pool:
            n = p["nx"] * p["ny"] * p["nz"]
            if chosen and total + n > budget:
                break
            chosen.append((p, i))
            total += n
        label = ENSEMBLE_DESC if name == "ensemble_64" else serve_desc(args, args.storage if args.storage != "f32"
                                                                        else "f16")
        return chosen, (f"FP64 oracle (plain C, OpenMP) on the {len(chosen)} smallest lattices of the {name} "
                        f"workload ({total} sites), one oracle step of each per benchmark step"), label
    params, init = WORKLOADS[name](storage="f32")
    n_full = params["nx"] * params["ny"] * params["nz"]
    if n_full <= budget or init["shape"] == 0:
        return [(params, init)], (f"FP64 oracle (plain C, OpenMP) on the full {params['nx']}x{params['ny']}x"
                                  f"{params['nz']} lattice of {name}, one oracle step per benchmark step"), \
            describe(name, params, args.storage)
    edge = int(max(8, min(params["nx"], ORACLE_CROP_EDGE, round(budget ** (1.0 / 3.0)))))
    scale = edge / params["nx"]
    p, i = droplet(edge, init["radius"] * scale, 1, rho_H=params["rho_H"])
    return [(p, i)], (f"FP64 oracle (plain C, OpenMP) on a {edge}^3 crop of the {name} workload (same geometry "
                      f"and parameters, radius scaled), one oracle step per benchmark step"), \
        describe(name, params, args.storage)


def run_reference(args):
    """The oracle arm: the FP64 plain-C oracle on the host cores, one oracle time step
    of a bounded sample of the workload per benchmark step (reference_lattices)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.workload == "ncomp3_128":
        rate, steps = ncomp_oracle_rate(max(5.0, min(120.0, 0.5 * (args.steps + args.warmup))))
        sample = (f"the N-component FP64 oracle (numpy, one thread) on the 24^3 three-component droplet of the "
                  f"same recipe (radius 4.5), {steps} steps")
        out = {"metric": "MLUPS", "value": rate, "unit": "MLUPS", "impl": "reference", "n_gpus": args.gpus,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": 24 ** 3 / rate / 1e3,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
               "data": "synthetic", "config": arm_config(args, world), "sample_sites": 24 ** 3,
               "cpu_baseline": {"value": rate, "unit": "MLUPS", "cores": 1, "kind": "oracle", "sample": sample},
               "e2e": {"value": rate, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(out))
        return
    lattices, sample, label = reference_lattices(args)
    cores = host_cores()
    oracle.set_threads(cores)
    ols = []
    for p, i in lattices:
        o = oracle.Lattice(p)
        o.init_shape(i)
        ols.append(o)
    for o in ols:
        o.step(args.warmup)
    t = time.perf_counter()
    for _ in range(args.steps):
        for o in ols:
            o.step(1)
    dt = time.perf_counter() - t
    n = sum(p["nx"] * p["ny"] * p["nz"] for p, _ in lattices)
    value = n * args.steps / dt / 1e6
    out = {"metric": "MLUPS", "value": value, "unit": "MLUPS", "impl": "reference", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": arm_config(args, world),
           "sample_sites": n,
           "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def oracle_sample(args, params, init):
    """The lattice the CPU baseline times: the workload's own lattice, or for a droplet
    larger than the crop-equivalent edge the 128^3 droplet of the same recipe (radius /
    box = 0.1875, same sink geometry and parameters); returns (params, init, words)."""
    from paper_1701_03637_gb300.workloads import droplet
    if init["shape"] == 0 or params["nx"] <= ORACLE_CROP_EDGE:
        return params, init, (f"the full {params['nx']}x{params['ny']}x{params['nz']} lattice of this workload")
    e = ORACLE_CROP_EDGE
    p, i = droplet(e, init["radius"] * e / params["nx"], 1, rho_H=params["rho_H"])
    return p, i, (f"the {e}^3 crop-equivalent droplet of this workload (same recipe: radius {i['radius']:g}, "
                  f"radius / box 0.1875, same sinks and parameters)")


def precision_record():
    """Error against the FP64 oracle of each storage type on the 128^3 crop-equivalent
    droplet, from the committed summary of the precision study
    (tests/test_gpu_precision.py): the 5000-step study when it is recorded, else the
    1000-step one; None when neither is."""
    fields = {kv.get("study"): kv for kv in profile_fields()}
    for study in ("precision_droplet_128_5000", "precision_droplet_128"):
        kv = fields.get(study)
        if kv is None:
            continue
        rec = {"source": f"profiles/{kv['file']}", "case": kv.get("case")}
        for st in ("f32", "f16", "bf16", "f16s"):
            if f"{st}_linf" in kv:
                rec[st] = {"density_linf": float(kv[f"{st}_linf"]), "density_l2": float(kv[f"{st}_l2"]),
                           "radius_error": float(kv[f"{st}_radius_error"])}
        return rec
    return None


def timed_steps(lat, steps, stream, barrier):
    """K steps between CUDA events on the launching stream, synchronized and behind a
    barrier on both sides; milliseconds."""
    import torch
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lat.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    return e0.elapsed_time(e1)


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_1701_03637_gb300 as sc

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    sc.build()

    def barrier():
        if world > 1:
            dist.barrier()

    def slowest(v):
        return max_over_ranks(v, world, "cuda")

    params, init = workload(args.workload, args.storage, args.tile, args.zchunk, args.layout, args.staging)
    n = params["nx"] * params["ny"] * params["nz"]
    aa = args.layout == "aa"
    need, free = sc.required_bytes(params), torch.cuda.mem_get_info()[0]
    if need > free:
        raise SystemExit(f"{args.workload} with {args.storage} populations and the {args.layout} layout needs "
                         f"{need / 1e9:.1f} GB of device memory, {free / 1e9:.1f} GB are free: use --layout aa "
                         f"(one population lattice) or --storage f16")
    lat = sc.Lattice(params)
    lat.init(init)
    tuned = None
    if not args.tile and not args.zchunk and not args.no_tune and not aa:
        tuned = lat.tune(trials=20)  # untimed; leaves the state unchanged (in place: nothing to tune)
    stream = torch.cuda.current_stream()
    lat.step(args.warmup)
    torch.cuda.synchronize()
    try:
        bus = torch.cuda.get_device_properties(local).pci_bus_id
    except Exception:
        bus = None
    sampler = ClockSampler()
    time.sleep(0.3)
    t0 = time.time()
    ms = timed_steps(lat, args.steps, stream, barrier)
    t1 = time.time()
    sampler.stop()
    ms_max = slowest(ms)
    d = lat.diagnostics()
    if d["status"] != 0:
        raise RuntimeError(f"diagnostics status {d['status']} after the timed run")
    launches = lat.launch_count(args.steps)

    value = replica_value(n, args.steps, world, ms_max)
    step_s = ms * 1e-3 / args.steps
    peak, peak_kind = measured_peak_hbm()
    achieved = BYTES_PER_SITE[args.storage] * n / step_s / 1e9
    info = lat.launch_info()
    tile_s = f"{info['tile_x']}x{info['tile_y']}"
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": profiled_traffic(args.workload, args.storage, tile_s, info["zchunk"], args.layout),
            "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback",
            "algorithmic_bytes_per_site": BYTES_PER_SITE[args.storage],
            "traffic_per": "time step (DRAM bytes of one step, as achieved is per step)",
            "kernel": lat.kernel_name(), "launches_per_step": launches / args.steps}

    # end to end through the public API: initial densities from pinned host memory,
    # the steps with FP64 diagnostics read back every 100 steps, final densities to host
    e2e = None
    if not args.no_e2e:
        rr0, rb0 = lat.read_fields()
        h_rr = torch.from_numpy(rr0.reshape(-1).copy()).pin_memory()
        h_rb = torch.from_numpy(rb0.reshape(-1).copy()).pin_memory()
        del rr0, rb0
        o_rr = torch.empty(n, dtype=torch.float32).pin_memory()
        o_rb = torch.empty(n, dtype=torch.float32).pin_memory()
        diag_every = 100
        barrier()
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        lat.init_fields_from(h_rr, h_rb)
        done = 0
        ndiag = 0
        while done < args.steps:
            k = min(diag_every, args.steps - done)
            lat.step(k)
            done += k
            lat.diagnostics()
            ndiag += 1
        lat.read_fields_into(o_rr, o_rb)
        torch.cuda.synchronize()
        w1 = time.perf_counter()
        barrier()
        wall = slowest(w1 - w0)
        diag_bytes = ndiag * lat.diag_bytes()
        e2e = {"value": n * args.steps * world / wall / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": 8 * n / args.steps,
               "d2h_bytes_per_step": (8 * n + diag_bytes) / args.steps,
               "includes": "init from pinned host densities, all steps, diagnostics every 100 steps, "
                           "final densities to pinned host"}
        del h_rr, h_rb, o_rr, o_rb

    # the other storage types on the same workload and layout (the precision study's
    # three runs), each timed over the same K steps after W warm-up steps
    variants = None
    if not args.no_variants and args.workload in DEFAULT_LAYOUT and args.storage == "f32":
        lat.close()
        variants = {}
        for st in ("f16", "bf16"):
            vp, vi = workload(args.workload, st, 0, 0, args.layout, args.staging)
            v = sc.Lattice(vp)
            v.init(vi)
            v.tune(trials=5)
            v.step(args.warmup)
            vms = slowest(timed_steps(v, args.steps, stream, barrier))
            vd = v.diagnostics()
            vval = replica_value(n, args.steps, world, vms)
            variants[st] = {"value": vval, "unit": "MLUPS", "ms_per_step": vms / args.steps,
                            "frac": BYTES_PER_SITE[st] * vval / world * 1e6 / 1e9 / peak,
                            "algorithmic_bytes_per_site": BYTES_PER_SITE[st], "status": vd["status"],
                            "radius": vd["radius"]}
            v.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = host_cores()
        op, oi, words = oracle_sample(args, params, init)
        rate, steps = oracle_rate(op, oi, 12.0, cores)
        rate1, steps1 = oracle_rate(op, oi, 6.0, 1)
        cpu = {"value": rate, "unit": "MLUPS", "cores": cores, "kind": "oracle",
               "sample": f"FP64 oracle (plain C, OpenMP, {cores} threads) on {words}, "
                         f"{steps} steps after its initial state",
               "single_thread": {"value": rate1, "unit": "MLUPS", "cores": 1,
                                 "sample": f"the same oracle on one thread, {steps1} steps"}}

    if rank == 0:
        clk = sampler.summary(t0, t1, bus)
        out = {"metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": args.storage, "data": "synthetic",
               "config": workload_config(args, params, world),
               "launch": dict({"tile": tile_s, "zchunk": info["zchunk"], "ctas": info["ctas"],
                               "staging": info["staging"], "autotuned": tuned is not None},
                              **({"bands": info["bands"]} if "bands" in info else {})),
               "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
               "clocks": clk, "diag": {k: d[k] for k in ("mass_r", "mass_b", "evaporated_mass", "radius")}}
        if variants is not None:
            out["storage_variants"] = variants
        rec = precision_record() if args.workload in DEFAULT_LAYOUT else None
        if rec is not None:
            out["error_vs_oracle"] = rec
        print(json.dumps(out))
    if variants is None:
        lat.close()
    if world > 1:
        dist.destroy_process_group()


def run_ensemble(args):
    """Batched ensemble of 64 lattices (edges log-uniform in [32, 96] per axis, films and
    droplets, g and tau drawn per lattice) advanced by one persistent launch per step,
    against the same lattices advanced one at a time through the single-lattice path."""
    import numpy as np
    import torch

    import torch.distributed as dist

    import paper_1701_03637_gb300 as sc
    from paper_1701_03637_gb300.workloads import ensemble, shard

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    sc.build()

    def barrier():
        if world > 1:
            dist.barrier()

    def slowest(v):
        return max_over_ranks(v, world, "cuda")

    # the 64 lattices are independent: each rank advances its share (no data exchange)
    everything = ensemble(64, 3, args.storage)
    all_sizes = [p["nx"] * p["ny"] * p["nz"] for p, _ in everything]
    n_all = sum(all_sizes)
    mine = shard(all_sizes, rank, world)
    members = [everything[k] for k in mine]
    sizes = [all_sizes[k] for k in mine]
    n = sum(sizes)
    arena = sum(sc.required_bytes(p) + 256 for p, _ in members) + (1 << 20)
    b = sc.Batch(arena, args.storage)
    lats = []
    for p, i in members:
        _, lat = b.add(p)
        lat.init(i)
        lats.append(lat)
    tile, zc = b.tune(trials=3)
    stream = torch.cuda.current_stream()
    b.step(args.warmup)
    torch.cuda.synchronize()
    sampler = ClockSampler()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    t0 = time.time()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    t1 = time.time()
    sampler.stop()
    ms = e0.elapsed_time(e1)  # this rank's launches (the roofline below is of its kernel)
    ms_max = slowest(ms)
    bad = [mine[k] for k, lat in enumerate(lats) if lat.diagnostics()["status"] != 0]
    nbad = int(round(sum_over_ranks(len(bad), world, "cuda")))
    value = n_all * args.steps / (ms_max * 1e-3) / 1e6
    peak, peak_kind = measured_peak_hbm()
    achieved = BYTES_PER_SITE[args.storage] * n / (ms * 1e-3 / args.steps) / 1e9

    # the same lattices one at a time (fresh copies), each through its own fused launches
    seq_steps = min(args.steps, 500)
    singles = []
    for p, i in members:
        g = sc.Lattice(p)
        g.init(i)
        g.step(2)
        singles.append(g)
    barrier()
    torch.cuda.synchronize()
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for g in singles:
        g.step(seq_steps)
    s1.record(stream)
    torch.cuda.synchronize()
    barrier()
    seq_ms = slowest(s0.elapsed_time(s1))
    seq_value = n_all * seq_steps / (seq_ms * 1e-3) / 1e6
    for g in singles:
        g.close()

    # end to end: densities of every member from pinned host memory, the steps with
    # every member's FP64 diagnostics read back every 100 steps, final densities to host
    host_in = [(torch.from_numpy(np.ascontiguousarray(lat.read_fields()[0]).reshape(-1)).pin_memory(),
                torch.from_numpy(np.ascontiguousarray(lat.read_fields()[1]).reshape(-1)).pin_memory()) for lat in lats]
    host_out = [(torch.empty(lat.n, dtype=torch.float32).pin_memory(),
                 torch.empty(lat.n, dtype=torch.float32).pin_memory()) for lat in lats]
    barrier()
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    for lat, (hr, hb) in zip(lats, host_in):
        lat.init_fields_from(hr, hb)
    done = ndiag = 0
    while done < args.steps:
        k = min(100, args.steps - done)
        b.step(k)
        done += k
        for lat in lats:
            lat.diagnostics()
        ndiag += 1
    for lat, (hr, hb) in zip(lats, host_out):
        lat.read_fields_into(hr, hb)
    torch.cuda.synchronize()
    wall = slowest(time.perf_counter() - w0)
    barrier()
    diag_bytes = sum_over_ranks(ndiag * sum(lat.diag_bytes() for lat in lats), world, "cuda")
    e2e = {"value": n_all * args.steps / wall / 1e6, "unit": "MLUPS", "h2d_bytes_per_step": 8 * n_all / args.steps,
           "d2h_bytes_per_step": (8 * n_all + diag_bytes) / args.steps,
           "includes": "init of all 64 members from pinned host densities, all steps, every member's "
                       "diagnostics every 100 steps, final densities to pinned host"}

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cores = host_cores()
        k = int(np.argmin(np.abs(np.asarray(sizes) - np.median(sizes))))
        rate, steps = oracle_rate(members[k][0], members[k][1], 12.0, cores)
        cpu = {"value": rate, "unit": "MLUPS", "cores": cores, "kind": "oracle",
               "sample": f"FP64 oracle on member {k} ({members[k][0]['nx']}x{members[k][0]['ny']}x"
                         f"{members[k][0]['nz']}, the median size), {steps} steps"}
    clk = sampler.summary(t0, t1)
    info = b.info()
    run_steps = 2000
    if rank != 0:
        b.close()
        dist.destroy_process_group()
        return
    out = {"metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
           # the 64 lattices are split over the ranks: the total work is fixed as N grows
           "scaling": "strong" if world > 1 else "weak",
           "vs_baseline": None, "dtype": args.storage, "data": "synthetic",
           "config": arm_config(args, world),
           "launch": {"tile": "%dx%d" % sc.tile_list()[tile - 1], "zchunk": zc, "items": info["items"],
                      "lattices_per_gpu": len(members)},
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                        "traffic": None, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                        "algorithmic_bytes_per_site": BYTES_PER_SITE[args.storage]},
           "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": args.steps + (args.steps + 31) // 32,
           "clocks": clk,
           "one_at_a_time": {"value": seq_value, "unit": "MLUPS", "steps": seq_steps,
                             "speedup_of_batch": value / seq_value},
           "runs_per_hour": {"batched": 64 * 3600.0 / (ms_max * 1e-3 / args.steps * run_steps),
                             "one_at_a_time": 64 * 3600.0 / (seq_ms * 1e-3 / seq_steps * run_steps),
                             "run": f"{run_steps} steps per lattice"},
           "members_with_bad_status": bad, "members_with_bad_status_all_ranks": nbad}
    print(json.dumps(out))
    b.close()
    if world > 1:
        dist.destroy_process_group()


def run_serve(args):
    """Served request stream: Poisson arrivals, cubic film/droplet lattices with edges
    log-uniform in [32, 160] and 2000-20000 steps, FP16-offset storage, continuous
    batching; against the same stream served one run at a time in plain FP32."""
    import numpy as np
    import torch

    import torch.distributed as dist

    import paper_1701_03637_gb300 as sc
    from paper_1701_03637_gb300.serve import Request, Server, dispatch, percentile, serve_one_at_a_time
    from paper_1701_03637_gb300.workloads import request_stream

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    sc.build()
    storage = args.storage if args.storage != "f32" else "f16"

    def served(reqs, run):
        """Every rank serves its round-robin share of the stream, starting together;
        the results of all ranks, in request order."""
        mine = dispatch(reqs, rank, world)
        if world > 1:
            dist.barrier()
        return gather_results(run(mine), world)

    def batched_server(cap=0, st=None):
        def run(mine):
            srv = Server(arena, st or storage, max_active_sites=cap)
            out = srv.run(mine)
            srv.close()
            return out
        return run

    def stream(count, rate, seed, st=None):
        return [Request(k, t, p, i, n) for k, (t, p, i, n) in
                enumerate(request_stream(count, rate, seed, storage=st or storage))]

    def summary(res, wall):
        lat = [r.latency for r in res]
        work = sum(r.sites * r.steps for r in res)
        return {"requests": len(res), "p50_latency_s": percentile(lat, 50), "p99_latency_s": percentile(lat, 99),
                "makespan_s": wall, "runs_per_hour": len(res) / wall * 3600.0, "mlups": work / wall / 1e6}

    arena = 24 << 30
    # warm-up: compile paths, first launches
    srv = Server(arena, storage)
    srv.run(stream(2, 1000.0, 99)[:2])
    srv.close()

    over = stream(args.requests, args.rate, 4)
    cap = 6 * 2 ** 20  # resident sites: about three 128^3 lattices, enough to fill the GPU
    sampler = ClockSampler()
    t0 = time.time()
    res = served(over, batched_server(cap))
    t1 = time.time()
    sampler.stop()
    batched = summary(res, max(r.finished for r in res))
    res_all = served(over, batched_server())
    uncapped = summary(res_all, max(r.finished for r in res_all))

    light = stream(max(4, args.requests // 4), args.light_rate, 5)
    res_light = served(light, batched_server(cap))
    light_s = summary(res_light, max(r.finished for r in res_light))
    light_work = sum(r.sites * r.steps for r in res_light)
    work_all = sum(r.sites * r.steps for r in res_all)

    # the same stream with FP16 of the scaled populations f / w (same relative spacing
    # in liquid and vapour), for its error against FP32
    scaled = stream(args.requests, args.rate, 4, "f16s")
    res_scaled = served(scaled, batched_server(cap, "f16s"))
    scaled_s = summary(res_scaled, max(r.finished for r in res_scaled))

    seq = served(over, lambda mine: serve_one_at_a_time(mine, "f32"))
    seq_s = summary(seq, max(r.finished for r in seq))

    def observable_errors(runs):
        """|final observable - FP32's| per run (interface position for films, radius for
        droplets, lattice units); FP32 matches the FP64 oracle to 1e-4 in density after
        1000 steps. Evicted runs have no final observable (counted in failed_runs)."""
        out = []
        for a, b in zip(runs, seq):
            if a.status or b.status:
                continue
            k = 1 if over[a.rid].init["shape"] == 0 else 2
            out.append(abs(a.series[-1][k] - b.series[-1][k]))
        return out

    errs = observable_errors(res)
    errs_scaled = observable_errors(res_scaled)
    failed = {"batched": sum(1 for r in res if r.status), "one_at_a_time_fp32": sum(1 for r in seq if r.status),
              "batched_scaled_f16": sum(1 for r in res_scaled if r.status)}
    clk = sampler.summary(t0, t1)
    work = sum(r.sites * r.steps for r in res)
    if rank != 0:
        dist.destroy_process_group()
        return
    out = {"metric": "MLUPS", "value": uncapped["mlups"], "unit": "MLUPS", "n_gpus": world, "steps": None,
           "warmup": 2, "ms_per_step": None, "higher_is_better": True,
           # one stream dispatched over the ranks: the total work is fixed as N grows
           "scaling": "strong" if world > 1 else "weak", "vs_baseline": None,
           "dtype": storage, "data": "synthetic",
           "config": arm_config(args, world),
           "launch": {"site_updates": work, "arena_bytes": arena},
           "serving": {"batched": uncapped,
                       "batched_site_cap": dict(batched, max_active_sites=cap),
                       # offered site updates per second (rate x mean work of a request) against
                       # what the batched server sustained: above 1 the queue still builds
                       "light_stream": dict(light_s, rate_per_s=args.light_rate,
                                            offered_vs_served=args.light_rate * light_work / len(light) / 1e6
                                            / uncapped["mlups"]),
                       "offered_vs_served": args.rate * work_all / len(over) / 1e6 / uncapped["mlups"],
                       "one_at_a_time_fp32": seq_s,
                       "failed_runs": failed,
                       "batched_scaled_f16": dict(scaled_s, max_active_sites=cap),
                       "observable_abs_error_vs_fp32": {
                           storage: {"max": max(errs, default=float("nan")), "median": percentile(errs, 50),
                                     "p99": percentile(errs, 99)},
                           "f16s": {"max": max(errs_scaled, default=float("nan")),
                                    "median": percentile(errs_scaled, 50), "p99": percentile(errs_scaled, 99)},
                           "what": "final interface position (films) or radius (droplets) of each served run "
                                   "against the same run in FP32, lattice units"}},
           "roofline": None, "cpu_baseline": None, "e2e": None, "gpu_launches": None, "clocks": clk}
    print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def run_slab(args):
    """One lattice of the workload split along z over the ranks (one slab per GPU,
    slab_ranges), every step exchanging the slabs' 2 boundary planes with the
    neighbouring ranks (NCCL; a single rank is its own neighbour) before the fused
    step: strong scaling, value = the whole lattice's site updates / the slowest
    rank's time."""
    import torch
    import torch.distributed as dist

    import paper_1701_03637_gb300 as sc
    from paper_1701_03637_gb300.slab import DistributedSlab, LocalSlabs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    sc.build()

    def barrier():
        if world > 1:
            dist.barrier()

    params, init = workload(args.workload, args.storage, args.tile, args.zchunk, "two")
    n = params["nx"] * params["ny"] * params["nz"]
    if world > 1:
        part = DistributedSlab(params)
        slab, stepper = part.slab, part
    else:
        part = LocalSlabs(params, 1)
        slab, stepper = part.slabs[0], part
    slab.init(init)
    stream = torch.cuda.current_stream()
    stepper.step(args.warmup)
    torch.cuda.synchronize()
    sampler = ClockSampler()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    t0 = time.time()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stepper.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    t1 = time.time()
    sampler.stop()
    ms = e0.elapsed_time(e1)
    ms_max = max_over_ranks(ms, world, "cuda")
    stepper.sync()
    d = slab.diagnostics()
    bad = sum_over_ranks(1.0 if d["status"] != 0 else 0.0, world, "cuda")
    own = params["nx"] * params["ny"] * (slab.z1 - slab.z0)
    value = n * args.steps / (ms_max * 1e-3) / 1e6
    peak, peak_kind = measured_peak_hbm()
    achieved = BYTES_PER_SITE[args.storage] * own / (ms * 1e-3 / args.steps) / 1e9
    if rank == 0:
        info = slab.launch_info()
        cfg = workload_config(args, params, world)
        out = {"metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
               "scaling": "strong", "vs_baseline": None, "dtype": args.storage, "data": "synthetic",
               "config": cfg,
               "launch": {"tile": f"{info['tile_x']}x{info['tile_y']}", "zchunk": info["zchunk"],
                          "ctas": info["ctas"], "staging": info["staging"], "slab_planes": slab.z1 - slab.z0},
               "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                            "frac": achieved / peak, "traffic": None,
                            "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                            "algorithmic_bytes_per_site": BYTES_PER_SITE[args.storage],
                            "note": "rank 0's step including its ghost exchange"},
               "cpu_baseline": None, "e2e": None, "gpu_launches": slab.launch_count(args.steps),
               "clocks": sampler.summary(t0, t1), "ranks_with_bad_status": bad}
        print(json.dumps(out))
    part.close()
    if world > 1:
        dist.destroy_process_group()


NCOMP_DESC = ("ncomp3_128: three-component D3Q19 Shan-Chen (Eq. (3) summed over the other components), 128^3 "
              "periodic, droplet of component 0 (radius 24, 0.7 / 0.04) in component 1, component 2 at 0.1 "
              "throughout, g01 = 3.6, g02 = g12 = 1.0, tau = 1, f32 populations, two lattices")


def ncomp_oracle_rate(budget_s):
    """The N-component FP64 oracle (numpy, as it stands) on a 24^3 sample of the
    ncomp3 recipe: MLUPS over whole-lattice steps, and the steps taken."""
    import numpy as np

    from oracle import multi
    from paper_1701_03637_gb300.workloads import three_component_droplet
    p, rho = three_component_droplet(24, 4.5, 1)
    o = multi.Lattice(p["nx"], p["ny"], p["nz"], p["tau"], p["g"])
    o.set_populations(multi.W[None, :, None, None, None] * rho[:, None].astype(np.float64))
    t = time.perf_counter()
    o.step(1)
    one = time.perf_counter() - t
    steps = max(1, int(budget_s / max(one, 1e-6)))
    t = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t
    return 24 ** 3 * steps / dt / 1e6, steps


def run_ncomp(args):
    """More than two components (sc_ncomp_*): three components at 128^3, one launch per
    step (tile columns marching plane chunks, Psi in a shared ring); independent
    replicas under torchrun."""
    import torch
    import torch.distributed as dist

    import paper_1701_03637_gb300 as sc
    from paper_1701_03637_gb300.ncomp import NLattice
    from paper_1701_03637_gb300.workloads import three_component_droplet

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    sc.build()

    def barrier():
        if world > 1:
            dist.barrier()

    params, rho = three_component_droplet(128, 24.0, 1)
    nc = len(params["tau"])
    n = params["nx"] * params["ny"] * params["nz"]
    lat = NLattice(**params)
    lat.init_fields(rho)
    lat.step(args.warmup)
    lat.sync()
    sampler = ClockSampler()
    time.sleep(0.3)
    t0 = time.time()
    ms = timed_steps(lat, args.steps, lat.stream, barrier)
    t1 = time.time()
    sampler.stop()
    ms_max = max_over_ranks(ms, world, "cuda")
    value = replica_value(n, args.steps, world, ms_max)
    peak, peak_kind = measured_peak_hbm()
    per_site = nc * BYTES_PER_SITE["f32"] // 2  # every population of every component read and written once
    achieved = per_site * n / (ms * 1e-3 / args.steps) / 1e9
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rate, steps = ncomp_oracle_rate(10.0)
        cpu = {"value": rate, "unit": "MLUPS", "cores": 1, "kind": "oracle",
               "sample": f"the N-component FP64 oracle (numpy, one thread) on the 24^3 three-component droplet "
                         f"of the same recipe (radius 4.5), {steps} steps"}
    if rank == 0:
        out = {"metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": arm_config(args, world),
               "launch": {"kernels": "k_n_step", "threads": 256, "components": nc},
               "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                            "frac": achieved / peak, "traffic": None,
                            "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                            "algorithmic_bytes_per_site": per_site,
                            "kernel": "k_n_step (one launch per step)"},
               "cpu_baseline": cpu, "e2e": None, "gpu_launches": args.steps,
               "clocks": sampler.summary(t0, t1)}
        print(json.dumps(out))
    lat.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "ncomp3_128":
        run_ncomp(args)
    elif args.layout == "slab":
        run_slab(args)
    elif args.workload == "ensemble_64":
        run_ensemble(args)
    elif args.workload == "serve":
        run_serve(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
