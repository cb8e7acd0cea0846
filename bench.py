"""Throughput of the fused Reg-FLBM D3Q27 step on GB300, one JSON line on stdout.

Workload (default): periodic 128^3 box, float32 populations, tau 0.8, rho0 1, kT 1e-4,
Philox seed 1, fluid at rest thermalised by the warm-up steps (the thermal-equilibrium
configuration of the paper's tests). One step = one launch of the fused
stream-and-collide kernel over every site. The two population buffers (2 x 226 MB)
exceed the 129 MB L2, so no flush is needed between steps.

Arms:
  --impl gb300 (default): the CUDA library through its C ABI; N > 1 ranks (torchrun)
      run independent replicas (weak scaling), barrier + max-over-ranks timing.
  --impl reference: the FP64 CPU oracle on the host cores, each step a bounded sample
      of sites of the same box, sized so the whole run ends within a few minutes.

Reported: MLUPS (sites x steps / s / 1e6) from CUDA events on the launching stream; the
roofline of the step kernel (216 algorithmic bytes per site update against the measured
HBM copy bandwidth); the end-to-end MLUPS through the ABI with host buffers; the
oracle's CPU MLUPS on a bounded sample; SM clocks sampled during the timed region.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Reg-FLBM D3Q27 MLUPS + % HBM roofline, FP32 vs mixed at fixed FDT error"
BYTES_PER_SITE = {"f32": 216, "f16": 108, "bf16": 108}  # 27 read + 27 written per site update
FALLBACK_HBM_GBS = 6800.0
PROFILES = os.path.join(ROOT, "profiles")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--edge", type=int, default=128)
    ap.add_argument("--tau", type=float, default=0.8)
    ap.add_argument("--kT", type=float, default=1e-4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--kernel", choices=["auto", "gather", "tma"], default="auto")
    ap.add_argument("--storage", choices=["f32", "f16", "bf16"], default="f32")
    ap.add_argument("--workload", choices=["box", "ensemble", "backtransform"], default="box",
                    help="one periodic box (default), the 64-replica ensemble of uneven sizes "
                         "advanced together (--storage applies), or the back transform of Eq. 11 "
                         "alone as float32 FMAs and as tensor-core MMA (a design measurement)")
    ap.add_argument("--tile", type=int, choices=[-1, 0, 96, 128, 192, 256, 512], default=0,
                    help="ensemble tile size for every replica (0: each row length its own, autotuned; "
                         "-1: by the order of preference, untimed)")
    ap.add_argument("--pattern", choices=["pingpong", "aa"], default="pingpong",
                    help="two population buffers (pull, ping-pong) or one updated in place (AA)")
    ap.add_argument("--init", choices=["rest", "taylor-green"], default="rest",
                    help="rest start, or the Taylor-Green vortex (u0 = 0.01, k = 2 pi / edge)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--decomp", choices=["none", "slab"], default="none",
                    help="none: every rank advances its own box (replicas); slab: the ranks hold "
                         "z-slabs of one periodic box of edge x edge x (edge * ranks) sites and "
                         "exchange their faces after every step (one rank: a slab periodic "
                         "through its own faces)")
    return ap.parse_args()


STORAGE_NAME = {"f32": "float32", "f16": "float16", "bf16": "bfloat16"}


def workload(args, world=1):
    e = args.edge
    nbuf = 1 if args.pattern == "aa" else 2
    nbytes = nbuf * 27 * BYTES_PER_SITE[args.storage] // 54 * e ** 3
    if getattr(args, "decomp", "none") == "slab":
        return {"workload": f"z-slabs of a periodic {e}x{e}x{e * world} Reg-FLBM D3Q27 box, one "
                            f"{e}^3 slab per rank, {STORAGE_NAME[args.storage]} populations, tau "
                            f"{args.tau}, rho0 1, kT {args.kT:g}, seed 1, rest start, faces exchanged "
                            "after every step",
                "init": args.init, "box": [e, e, e * world], "sites": e ** 3 * world, "tau": args.tau,
                "kT": args.kT, "storage": f"{args.storage} shifted by w_i rho0",
                "streaming": "pull, ping-pong" if nbuf == 2 else "AA, one buffer in place",
                "l2": f"inputs {nbytes / 1e6:.0f} MB per rank > 129 MB L2, no flush"
                      if nbytes > 129e6 else f"inputs {nbytes / 1e6:.0f} MB per rank fit in the 129 MB L2",
                "parallelism": "z-slabs" if world > 1 else "one z-slab, periodic through its own faces"}
    return {"workload": f"periodic {e}^3 Reg-FLBM D3Q27 thermal equilibrium, "
                        f"{STORAGE_NAME[args.storage]} populations, tau {args.tau}, rho0 1, "
                        f"kT {args.kT:g}, seed 1, "
                        + ("rest start" if args.init == "rest" else "Taylor-Green u0 0.01 start"),
            "init": args.init, "box": [e, e, e], "sites": e ** 3, "tau": args.tau, "kT": args.kT,
            "storage": f"{args.storage} shifted by w_i rho0",
            "streaming": "pull, ping-pong" if nbuf == 2 else "AA, one buffer in place",
            "l2": f"inputs {nbytes / 1e6:.0f} MB ({nbuf} population buffer{'s' if nbuf == 2 else ''})"
                  + (" > 129 MB L2, no flush" if nbytes > 129e6 else " fit in the 129 MB L2"),
            "parallelism": "replicas"}


# ------------------------------------------------------------------ measurement helpers
def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            peaks = json.load(fh)
        return float(peaks["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# the sources the ping-pong TMA step kernel is compiled from (its translation unit and
# every header it includes)
STEP_KERNEL_SOURCES = ("collide.cuh", "d3q27.cuh", "philox.cuh", "rflbm_internal.h",
                       "rflbm_step_tma.cu", "rflbm_step_tma16.cu", "step_tma.cuh", "storage.cuh",
                       "tma.cuh")
AA_KERNEL_SOURCES = STEP_KERNEL_SOURCES + ("step_aa.cuh", "rflbm_step_aa_f32.cu", "rflbm_step_aa_f16.cu",
                                           "rflbm_step_aa_bf16.cu")
BATCH_KERNEL_SOURCES = ("collide.cuh", "d3q27.cuh", "philox.cuh", "rflbm_internal.h", "storage.cuh", "tma.cuh",
                        "rflbm_aux.h", "rflbm_batch.cu")


def strip_comments(src):
    """C/C++ source without its comments and blank lines (string and character literals
    kept), so that the hash below changes with the code only."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return "\n".join(line.rstrip() for line in "".join(out).splitlines() if line.strip())


def kernel_source_hash(names=STEP_KERNEL_SOURCES):
    """Hash of the code (comments excluded) the step kernels are compiled from."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2507_08820_gb300", "csrc")
    for name in names:
        with open(os.path.join(csrc, name), encoding="utf-8") as fh:
            h.update((name + strip_comments(fh.read())).encode())
    return h.hexdigest()[:16]


def kernel_name(kind, path, kT, model, storage="f32", pattern="pingpong", sites_per_thread=1,
                odd_sites_per_thread=None):
    """(name, profile stem) of the step kernel; for AA, sites_per_thread is that of the
    even steps and odd_sites_per_thread that of the odd steps (default: the same). The stem
    of a kernel without noise or of the BGK model carries a suffix, so that it never reads
    the profile of the Reg-FLBM fluctuating kernel."""
    name, stem = _kernel_name(kind, path, kT, model, storage, pattern, sites_per_thread, odd_sites_per_thread)
    return name, stem + ("" if kT > 0 else "_kt0") + ("_bgk" if model else "")


def _kernel_name(kind, path, kT, model, storage, pattern, sites_per_thread, odd_sites_per_thread):
    noise = "noise" if kT > 0 else "no noise"
    m = "BGK" if model else "Reg"
    if pattern == "aa":
        if kind == 2:
            odd = sites_per_thread if odd_sites_per_thread is None else odd_sites_per_thread
            even_k = "step_aa_even_pair" if sites_per_thread == 2 else "step_aa_even"
            odd_k = "step_aa_odd_pair" if odd == 2 else "step_aa_odd"
            tag = {(1, 1): "", (2, 2): "pair_", (1, 2): "oddpair_", (2, 1): "evenpair_"}[(sites_per_thread, odd)]
            return f"{even_k}+{odd_k}<{storage}, {path}, {m}, {noise}>", f"step_aa_{tag}{storage}_{path}"
        return f"step_aa_gather<{storage}, {m}, {noise}>", f"step_aa_gather_{storage}"
    if kind == 2 and sites_per_thread == 2:
        return f"step_tma_pair<{storage}, {path}, {m}, {noise}>", f"step_tma_pair_{storage}_{path}"
    if kind == 2:
        return f"step_tma<{storage}, {path}, {m}, {noise}>", f"step_tma_{storage}_{path}"
    return f"step_pull<{storage}, {m}, {noise}>", f"step_pull_{storage}"


def profiled_traffic(profile_stem, edge):
    """DRAM bytes per launch of the step kernel (per step of an ensemble: all its launches) from the committed ncu summary
    (<stem>_<edge>cubed.md, or <stem>_<edge>.md when edge is a workload name), or None when
    the summary is missing or was taken on different kernel sources."""
    suffix = f"{edge}cubed" if isinstance(edge, int) else edge
    try:
        text = open(os.path.join(PROFILES, f"{profile_stem}_{suffix}.md")).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_(?:launch|step):\s*([0-9.eE+]+)\s*\(sources ([0-9a-f]+)\)", text)
    names = (AA_KERNEL_SOURCES if profile_stem.startswith("step_aa") else
             BATCH_KERNEL_SOURCES if profile_stem.startswith("k_batch") else STEP_KERNEL_SOURCES)
    if not m or m.group(2) != kernel_source_hash(names):
        return None
    return float(m.group(1))


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while the timed region runs."""

    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.uuid = uuid
        self.proc = None
        self.path = os.path.join("/tmp", f"rflbm_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            if self.uuid and parts[0] != self.uuid:
                continue
            rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "samples": 0, "reasons": []}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = sorted(x for x in (num(r[1]) for r in rows) if x is not None)
        mx = [x for x in (num(r[2]) for r in rows) if x is not None]
        pw = [x for x in (num(r[3]) for r in rows) if x is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "samples": len(rows), "reasons": reasons}


def device_uuid(torch):
    try:
        u = str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


# ------------------------------------------------------------------ CPU oracle timing
# One oracle worker: imports, calibrates its per-site cost, waits for the common start
# time, then collides and streams its own chunk of the box's sites (every `workers`-th site,
# starting at its index) for the given number of steps in one thread.
_ORACLE_WORKER = r"""
import json, sys, time
cfg = json.loads(sys.argv[1])
sys.path.insert(0, cfg["root"])
import numpy as np
from oracle import rflbm_oracle as o
from paper_2507_08820_gb300 import workloads as W
n, k, workers = cfg["edge"] ** 3, cfg["index"], cfg["workers"]
f = o.rest_state(512) + W.population_perturbation(512, 3, 1e-4)
t0 = time.perf_counter(); o.collide(f, cfg["tau"], cfg["kT"], 1, 0, np.arange(512, dtype=np.uint64))
per_site = (time.perf_counter() - t0) / 512
chunk = np.arange(k, n, workers, dtype=np.int64)
steps = cfg["steps"] or 2  # None: at least two steps, more while the budget allows
m = int(cfg["budget"] / steps / per_site)
m = max(min(cfg["min_sites"], chunk.size), min(m, chunk.size))
if not cfg["steps"]:
    steps = max(2, int(cfg["budget"] / (m * per_site)))
sites = chunk[:m]
f = o.rest_state(sites.size) + W.population_perturbation(sites.size, 5 + k, 1e-4)
while time.time() < cfg["t_go"]:
    time.sleep(0.005)
t0 = time.time()
for t in range(steps):
    fs = o.collide(f, cfg["tau"], cfg["kT"], 1, t, sites.astype(np.uint64))
    f = o.stream(fs, (sites.size, 1, 1))
t1 = time.time()
print(json.dumps(dict(sites=int(sites.size), steps=steps, t0=t0, t1=t1)))
"""


def host_cores():
    """Host cores this process may use (the affinity mask where the OS reports one)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sample_rate(edge, tau, kT, budget_s, steps, workers=None, min_sites=16):
    """Times the FP64 oracle's per-site collision plus streaming on a bounded sample of the
    box's sites, on every host core: one single-threaded worker process per core, each on
    its own chunk of sites (every `workers`-th site), all starting at one agreed wall-clock
    time. Each worker's sample is sized so that its `steps` steps take about `budget_s`
    seconds (steps=None: at least two, more while the budget allows). Returns dict(mlups,
    sites, steps, seconds, workers): site updates of all workers over the wall time from
    the first start to the last finish."""
    workers = workers or host_cores()
    t_go = time.time() + 3.0 + 0.2 * workers  # after every worker's imports and calibration
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    procs = []
    for k in range(workers):
        cfg = dict(root=ROOT, edge=edge, tau=tau, kT=kT, budget=budget_s, steps=steps, index=k,
                   workers=workers, min_sites=min_sites, t_go=t_go)
        procs.append(subprocess.Popen([sys.executable, "-c", _ORACLE_WORKER, json.dumps(cfg)],
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env))
    results = []
    for p in procs:
        out, err = p.communicate(timeout=max(600, 20 * budget_s))
        if p.returncode != 0:
            raise RuntimeError("oracle timing failed:\n" + err[-2000:])
        results.append(json.loads(out.strip().splitlines()[-1]))
    wall = max(r["t1"] for r in results) - min(r["t0"] for r in results)
    updates = sum(r["sites"] * r["steps"] for r in results)
    return dict(mlups=updates / wall / 1e6, sites=sum(r["sites"] for r in results),
                steps=max(r["steps"] for r in results), seconds=wall, workers=workers)


def cpu_baseline_entry(r, edge, per_step):
    """The cpu_baseline object of a JSON line from an oracle_sample_rate result."""
    return {"value": r["mlups"], "unit": "MLUPS", "cores": r["workers"], "nproc": os.cpu_count(),
            "kind": "oracle",
            "sample": f"FP64 oracle collision + streaming of {r['sites']} sampled sites of the "
                      f"{edge}^3 box{' per step' if per_step else ''}, {r['steps']} steps, "
                      f"{r['seconds']:.1f} s, {r['workers']} single-threaded processes "
                      f"(one per host core, each on its own chunk of sites)"}


# ------------------------------------------------------------------ reference arm
def reference_arm(args):
    from paper_2507_08820_gb300 import dist
    info = dist.rank_info()
    if info.rank != 0:
        return 0
    # each of the warmup + steps "steps" collides a bounded sample of the box's sites on
    # every host core; the whole run is held to about two minutes
    total = max(1, args.steps + args.warmup)
    r = oracle_sample_rate(args.edge, args.tau, args.kT, budget_s=min(120.0, 2.0 * total), steps=total)
    line = {
        "impl": "reference", "metric": METRIC, "value": r["mlups"], "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * r["seconds"] / r["steps"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload(args),
        "cpu_baseline": cpu_baseline_entry(r, args.edge, True),
        "e2e": {"value": r["mlups"], "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ GPU arm
def time_steps(R, torch, box, stream, steps, exchange=None):
    """CUDA-event time (ms) of `steps` steps on the box's stream; with `exchange`, a z-slab
    that exchanges its faces (exchange()) after every step."""
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    advance(R, box, steps, exchange)
    end.record(stream)
    end.synchronize()
    return start.elapsed_time(end)


def advance(R, box, steps, exchange=None):
    if exchange is None:
        R.rflbm_step(box.h, steps)
        return
    for _ in range(steps):
        R.rflbm_step(box.h, 1)
        exchange()


def slab_rings(R, torch, args, peak, sizes=(2, 4)):
    """K z-slabs of one periodic edge x edge x (K edge) box on this GPU, one edge^3 slab each,
    on one stream, their faces exchanged by rflbm_slab_exchange after every step: the cost
    of the decomposition with real neighbours, without the link between GPUs."""
    storage = {"f32": R.RFLBM_STORE_F32, "f16": R.RFLBM_STORE_F16, "bf16": R.RFLBM_STORE_BF16}[args.storage]
    pattern = {"pingpong": R.RFLBM_PATTERN_PINGPONG, "aa": R.RFLBM_PATTERN_AA}[args.pattern]
    e = args.edge
    steps = max(20, min(args.steps, 500))
    out = {}
    for k in sizes:
        stream = torch.cuda.Stream()
        slabs = [R.Box(e, e, e, tau=args.tau, kT=args.kT, seed=1, stream=stream.cuda_stream, storage=storage,
                       pattern=pattern, z0=i * e, nz_global=k * e) for i in range(k)]
        for b in slabs:
            R.rflbm_init_rest(b.h)
        hs = [b.h for b in slabs]

        def step():
            for b in slabs:
                R.rflbm_step(b.h, 1)
            R.rflbm_slab_exchange(hs)
        for _ in range(10):
            step()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(steps):
            step()
        ev1.record(stream)
        ev1.synchronize()
        ms = ev0.elapsed_time(ev1) / steps
        sites = k * e ** 3
        out[str(k)] = {"slabs": k, "box": [e, e, k * e], "steps": steps, "ms_per_step": ms,
                       "value": sites / (ms * 1e-3) / 1e6, "unit": "MLUPS",
                       "roofline_frac": BYTES_PER_SITE[args.storage] * sites / (ms * 1e-3) / 1e9 / peak}
        for b in slabs:
            b.close()
    return out


def ensemble_arm(args):
    """The 64-replica ensemble (edges 16-96, seeds 1..64, kT log-uniform in [1e-5, 1e-3],
    tau uniform in [0.55, 1.2]) advanced together: MLUPS over all replicas, one CUDA graph
    of per-step launches per call."""
    import torch

    from paper_2507_08820_gb300 import build, dist
    from paper_2507_08820_gb300 import workloads as W
    build.build()
    from paper_2507_08820_gb300 import rflbm as R

    info = dist.rank_info()
    torch.cuda.set_device(info.local_rank)
    dev = torch.device("cuda", info.local_rank)
    dist.init(info, "nccl")
    storage = {"f32": R.RFLBM_STORE_F32, "f16": R.RFLBM_STORE_F16, "bf16": R.RFLBM_STORE_BF16}[args.storage]
    reps = W.replica_ensemble(64, seed=0)
    sites = sum(r["nx"] * r["ny"] * r["nz"] for r in reps)
    bh = R.rflbm_batch_create(reps, storage=storage, tile=args.tile)
    R.rflbm_batch_init_rest(bh)
    R.rflbm_batch_run(bh, args.warmup)
    R.rflbm_batch_prepare(bh, args.steps)  # the timed call's graph is built before the timed region
    R.rflbm_batch_synchronize(bh)
    sampler = ClockSampler(device_uuid(torch))
    dist.barrier(info, info.local_rank)
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(torch.cuda.default_stream())
    R.rflbm_batch_run(bh, args.steps)
    ev1.record(torch.cuda.default_stream())
    ev1.synchronize()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    dist.barrier(info, info.local_rank)
    ms_max = dist.max_over_ranks(info, ms, dev)
    tile, per_sm, tiles = R.rflbm_batch_tuning(bh)
    launches = R.rflbm_batch_launches_per_step(bh) * args.steps
    tilings = [R.rflbm_batch_replica_tiling(bh, r) for r in range(len(reps))]
    R.rflbm_batch_destroy(bh)
    # the row-tile kernels of a step, by tile size, with the share of the sites each updates
    row_sites = {}
    for (t, rows), r in zip(tilings, reps):
        if rows:
            row_sites[t] = row_sites.get(t, 0) + r["nx"] * r["ny"] * r["nz"]
    kname = ("k_batch_step<{}, {}, rows>" if args.storage == "f32" else "k_batch_rows_pair<{}, {}>")
    kernels = " + ".join(kname.format(args.storage, t) for t in sorted(row_sites))
    site_share = {str(t): row_sites[t] / sites for t in sorted(row_sites)}
    stem = ("k_batch_step_" if args.storage == "f32" else "k_batch_rows_pair_") + args.storage + "_" + (
        str(tile) if tile > 0 else "per_replica")
    if info.rank != 0:
        dist.finalize(info)
        return 0
    bps = BYTES_PER_SITE[args.storage]
    achieved = bps * sites * args.steps / (ms * 1e-3) / 1e9
    peak, peak_kind = measured_peak()
    line = {
        "metric": METRIC, "value": info.world * sites * args.steps / (ms_max * 1e-3) / 1e6, "unit": "MLUPS",
        "n_gpus": info.world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "storage_dtype": args.storage, "data": "synthetic",
        "config": {"workload": f"64-replica Reg-FLBM ensemble, edges 16-96, {STORAGE_NAME[args.storage]} "
                               "populations, rest start", "replicas": len(reps), "sites": sites,
                   "tile": tile if tile > 0 else ("autotuned per row length" if tile == 0 else
                                                  "per row length, untimed"),
                   "row_tile_site_share": site_share,
                   "ctas_per_sm": per_sm, "tiles_per_step": tiles,
                   "parallelism": "replicas"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": f"hbm_gbs of {peak_kind}",
                     "traffic": profiled_traffic(stem, "ensemble64"),
                     "kernel": kernels, "launches_per_step": launches // args.steps,
                     "algorithmic_bytes_per_step": bps * sites},
        "cpu_baseline": None, "e2e": None, "gpu_launches": launches, "clocks": clocks,
    }
    print(json.dumps(line))
    dist.finalize(info)
    return 0


def init_taylor_green(R, torch, box, e, dev, u0=0.01):
    """The Taylor-Green vortex u0 (-cos kx sin ky, sin kx cos ky, 0), k = 2 pi / e, with its
    incompressible pressure as density (the workloads module's fields), built on the device
    (the host would need 4 N doubles) and loaded as the equilibrium of Eq. 26."""
    import numpy as np
    k = 2.0 * np.pi / e
    x = torch.arange(e, dtype=torch.float64, device=dev)
    cx, sx = torch.cos(k * x), torch.sin(k * x)
    u = torch.zeros((3, e, e, e), dtype=torch.float64, device=dev)  # (3, z, y, x)
    u[0] = -u0 * (cx[None, None, :] * sx[None, :, None])
    u[1] = u0 * (sx[None, None, :] * cx[None, :, None])
    c2 = torch.cos(2 * k * x)
    rho = 1.0 - u0 ** 2 * 3.0 / 4.0 * (c2[None, None, :] + c2[None, :, None]).expand(e, e, e)
    rho = rho.contiguous()
    R.rflbm_init_field(box.h, rho, u)
    torch.cuda.synchronize()
    del u, rho
    torch.cuda.empty_cache()


def time_variant(R, torch, stream, shape, k, peak, bps, init="rest", warm=3, **kw):
    """MLUPS and roofline fraction of one configuration: a box of its own (freed before the
    next), `warm` untimed steps (the first AA step reveals the odd-step form), then k steps
    timed with CUDA events on the launching stream."""
    e = shape[0]
    vb = R.Box(*shape, tau=kw.pop("tau", 0.8), seed=1, stream=stream.cuda_stream, **kw)
    try:
        if init == "rest":
            R.rflbm_init_rest(vb.h)
        else:
            init_taylor_green(R, torch, vb, e, torch.device("cuda", torch.cuda.current_device()))
        kind, path = R.rflbm_step_path(vb.h)
        pairs = R.rflbm_step_sites_per_thread(vb.h)
        R.rflbm_step(vb.h, 1)
        odd_pairs = R.rflbm_step_sites_per_thread(vb.h)
        R.rflbm_step(vb.h, max(0, warm - 1))
        R.rflbm_synchronize(vb.h)
        vms = time_steps(R, torch, vb, stream, k)
        st, status = R.rflbm_stats(vb.h)
        n = vb.n
        pattern = "aa" if kw.get("pattern") == R.RFLBM_PATTERN_AA else "pingpong"
        storage = {R.RFLBM_STORE_F32: "f32", R.RFLBM_STORE_F16: "f16",
                   R.RFLBM_STORE_BF16: "bf16"}[kw.get("storage", R.RFLBM_STORE_F32)]
        kname, _ = kernel_name(kind, path, kw.get("kT", 0.0), kw.get("model", 0), storage, pattern,
                               pairs, odd_pairs)
        sites_s = n * k / (vms * 1e-3)
        return {"value": sites_s / 1e6, "unit": "MLUPS", "steps": k, "box": list(shape),
                "ms_per_step": vms / k, "roofline_frac": bps * sites_s / 1e9 / peak,
                "bytes_per_site": bps, "kernel": kname, "init": init,
                "finite_after": bool(status == R.RFLBM_OK)}
    finally:
        vb.close()
        torch.cuda.synchronize()
        torch.cuda.empty_cache()


def storage_accuracy(R, torch, stream, edge=128, steps=20, tau=0.8, kT=1e-4):
    """Error of each storage format "at fixed FDT error": from the same thermal initial
    state (rflbm_init_thermal draws it identically in every format), `steps` steps of each
    format; rho, u and Pi of every site against the float32 run, as RMS and maximum in units
    of each field's thermal standard deviation (float32 itself is within 2.2e-7 RMS of the
    FP64 oracle in the parity tests), the largest deviation of the 27 per-site mode
    variances from the fluctuation-dissipation value rho0 kT b_k / cs2 (Sec. II.A), and the
    static structure factors S(k) of rho, rho u and Pi (shell bands 4-8, 8-16, 16-32 of
    |k| L / 2 pi): their largest deviation from the flat values of Sec. III (rho0 kT / cs2
    for rho, rho0 kT for rho u, 2 rho0 kT cs2 and rho0 kT cs2 for the diagonal and
    off-diagonal Pi), and of each 16-bit format's bands from float32's."""
    import numpy as np
    n = edge ** 3
    dev = torch.device("cuda", torch.cuda.current_device())
    cs2 = 1.0 / 3.0
    # thermal standard deviations of rho, u_a, Pi_aa, Pi_ab at rho0 = 1
    sd = [np.sqrt(kT / cs2)] + [np.sqrt(kT)] * 3 + [np.sqrt(2 * kT * cs2)] * 3 + [np.sqrt(kT * cs2)] * 3
    fields, out, sk_bands = {}, {}, {}
    for name, st in (("f32", R.RFLBM_STORE_F32), ("f16", R.RFLBM_STORE_F16), ("bf16", R.RFLBM_STORE_BF16)):
        box = R.Box(edge, edge, edge, tau=tau, kT=kT, seed=1, stream=stream.cuda_stream, storage=st)
        R.rflbm_init_thermal(box.h)
        R.rflbm_step(box.h, steps)
        rho = torch.empty(n, dtype=torch.float64, device=dev)
        u = torch.empty((3, n), dtype=torch.float64, device=dev)
        pi = torch.empty((6, n), dtype=torch.float64, device=dev)
        R.rflbm_moments(box.h, rho, u, pi)
        s1, s2 = R.rflbm_mode_sums(box.h)
        ns = R.rflbm_shell_count(box.h)
        bands, band_sd = [], None
        for f in range(10):
            sk, count = R.rflbm_structure_factor(box.h, f, ns)
            bands.append([sk[lo:hi].sum() / count[lo:hi].sum() for lo, hi in ((4, 8), (8, 16), (16, 33))])
            # one snapshot: S of a real Gaussian field is exponential on half of the vectors
            band_sd = [float(np.sqrt(2.0 / count[lo:hi].sum())) for lo, hi in ((4, 8), (8, 16), (16, 33))]
        box.close()
        bands = np.array(bands)
        var = s2 / n - (s1 / n) ** 2
        ratio = var / (kT * mode_norms() / cs2)
        fields[name] = torch.cat([rho[None], u, pi])
        s_theory = np.array([kT / cs2] + [kT] * 3 + [2 * kT * cs2] * 3 + [kT * cs2] * 3)
        sk_bands[name] = bands
        entry = {"fdt_mode_variance_max_dev": float(np.max(np.abs(ratio - 1.0))),
                 "fdt_mode_variance_mean": float(np.mean(ratio)),
                 "sk_max_dev_from_theory": float(np.max(np.abs(bands / s_theory[:, None] - 1.0))),
                 "sk_band_sampling_rel_sd": band_sd}
        if name != "f32":
            entry["sk_max_rel_diff_vs_f32"] = float(np.max(np.abs(bands / sk_bands["f32"] - 1.0)))
        if name != "f32":
            d = (fields[name] - fields["f32"]).abs() / torch.tensor(sd, dtype=torch.float64, device=dev)[:, None]
            entry["vs_f32_rms_in_thermal_sd"] = float(torch.sqrt((d * d).mean()))
            entry["vs_f32_max_in_thermal_sd"] = float(d.max())
        out[name] = entry
        del rho, u, pi
    del fields
    torch.cuda.empty_cache()
    return {"workload": f"{edge}^3 thermal initial state, tau {tau}, kT {kT:g}, {steps} steps, seed 1",
            "fields": "rho, u, Pi per site; S(k) of rho, rho u, Pi in shell bands 4-8, 8-16, 16-32", **out}


def mode_norms():
    """b_k of the 27 modes of Table II (products of the 1-D norms 1, 1/3, 2/9 over the
    Hermite exponents of each mode, in the order rflbm_mode_sums reports)."""
    import numpy as np
    beta = (1.0, 1.0 / 3.0, 2.0 / 9.0)
    # Table II order: exponent triples (p, q, r) per mode k
    pqr = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (0, 2, 0), (0, 0, 2), (1, 1, 0),
           (1, 0, 1), (0, 1, 1), (2, 1, 0), (2, 0, 1), (1, 2, 0), (1, 0, 2), (0, 1, 2), (0, 2, 1),
           (1, 1, 1), (2, 2, 0), (2, 0, 2), (0, 2, 2), (1, 1, 2), (1, 2, 1), (2, 1, 1), (2, 1, 2),
           (2, 2, 1), (1, 2, 2), (2, 2, 2)]
    return np.array([beta[p] * beta[q] * beta[r] for p, q, r in pqr])


def gb300_arm(args):
    import numpy as np
    import torch

    from paper_2507_08820_gb300 import build, dist
    build.build()
    from paper_2507_08820_gb300 import rflbm as R

    info = dist.rank_info()
    torch.cuda.set_device(info.local_rank)
    dev = torch.device("cuda", info.local_rank)
    dist.init(info, "nccl")
    e = args.edge
    n = e ** 3
    stream = torch.cuda.Stream(device=dev)
    kernel = {"auto": R.RFLBM_KERNEL_AUTO, "gather": R.RFLBM_KERNEL_GATHER,
              "tma": R.RFLBM_KERNEL_TMA}[args.kernel]
    storage = {"f32": R.RFLBM_STORE_F32, "f16": R.RFLBM_STORE_F16, "bf16": R.RFLBM_STORE_BF16}
    pattern = {"pingpong": R.RFLBM_PATTERN_PINGPONG, "aa": R.RFLBM_PATTERN_AA}[args.pattern]
    slab = args.decomp == "slab"
    exchange = None
    if slab:
        # rank r: rows r e .. (r + 1) e - 1 of one box; replica word 0 for every rank (one box)
        z0, nz = dist.slab_bounds(e * info.world, info.world, info.rank)
        box = R.Box(e, e, nz, tau=args.tau, kT=args.kT, seed=1, stream=stream.cuda_stream,
                    torch_buffers=True, device=info.local_rank, kernel=kernel,
                    storage=storage[args.storage], pattern=pattern, z0=z0, nz_global=e * info.world)
        side = torch.cuda.Stream(device=dev)
        if info.world == 1:
            exchange = lambda: R.rflbm_slab_exchange([box.h])  # noqa: E731
        else:
            exchange = lambda: dist.exchange_slab(R, box, info, side)  # noqa: E731
    else:
        box = R.Box(e, e, e, tau=args.tau, kT=args.kT, seed=1, replica=info.rank,
                    stream=stream.cuda_stream, torch_buffers=True, device=info.local_rank,
                    kernel=kernel, storage=storage[args.storage], pattern=pattern)
    if args.init == "rest":
        R.rflbm_init_rest(box.h)
    else:
        init_taylor_green(R, torch, box, e, dev)
    kind, path = R.rflbm_step_path(box.h)
    pairs = R.rflbm_step_sites_per_thread(box.h)
    odd_pairs = pairs
    warm = args.warmup
    if args.pattern == "aa" and warm > 0:  # the odd AA steps may run the other form
        advance(R, box, 1, exchange)
        odd_pairs = R.rflbm_step_sites_per_thread(box.h)
        warm -= 1
    R.rflbm_synchronize(box.h)

    sampler = ClockSampler(device_uuid(torch))
    sampler.start()
    time.sleep(0.3)  # let the sampler take its first reading
    # the warm-up steps run directly before the timed region, so that the GPU enters it busy
    advance(R, box, warm, exchange)
    R.rflbm_synchronize(box.h)
    dist.barrier(info, info.local_rank)
    torch.cuda.synchronize()
    ms = time_steps(R, torch, box, stream, args.steps, exchange)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    dist.barrier(info, info.local_rank)
    ms_max = dist.max_over_ranks(info, ms, dev)
    launches = R.rflbm_launches_per_step(box.h) * args.steps
    st, status = R.rflbm_stats(box.h)

    # end to end through the ABI with host buffers: every step imports the populations from
    # page-locked host memory, steps, and exports the step's result (the populations) back
    e2e = None
    if not args.no_e2e:
        k_e2e = max(3, min(args.steps, 2000) // 10)
        host_in = torch.empty((27, n), dtype=torch.float32).pin_memory()
        host_out = torch.empty((27, n), dtype=torch.float32).pin_memory()
        R.rflbm_get_populations_f32(box.h, host_in)
        R.rflbm_set_populations_f32(box.h, host_in)   # untimed: allocates the staging buffer
        dist.barrier(info, info.local_rank)
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            R.rflbm_set_populations_f32(box.h, host_in)
            advance(R, box, 1, exchange)
            R.rflbm_get_populations_f32(box.h, host_out)
        e2e_s = dist.max_over_ranks(info, time.perf_counter() - t0, dev)
        e2e = {"value": info.world * n * k_e2e / e2e_s / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": 27 * 4 * n, "d2h_bytes_per_step": 27 * 4 * n, "steps": k_e2e,
               "path": "rflbm_set_populations_f32 (pinned host) + rflbm_step + "
                       "rflbm_get_populations_f32 (pinned host)"}
        del host_in, host_out

    variants = {}
    accuracy = None
    if not args.no_variants and info.world == 1 and not slab:
        peak_v, _ = measured_peak()
        st_main = storage[args.storage]
        k = max(10, args.steps // 4)
        F32, F16, BF16, AA = R.RFLBM_STORE_F32, R.RFLBM_STORE_F16, R.RFLBM_STORE_BF16, R.RFLBM_PATTERN_AA
        for name, shape, init, kw, bps in (
                ("reg_lbm_kT0", (e, e, e), "rest", dict(kT=0.0, storage=st_main), BYTES_PER_SITE[args.storage]),
                ("bgk_flbm", (e, e, e), "rest", dict(kT=args.kT, model=R.RFLBM_MODEL_BGK, storage=st_main),
                 BYTES_PER_SITE[args.storage]),
                ("f16_reg_flbm", (e, e, e), "rest", dict(kT=args.kT, storage=F16), 108),
                ("f16_reg_lbm_kT0", (e, e, e), "rest", dict(kT=0.0, storage=F16), 108),
                ("bf16_reg_flbm", (e, e, e), "rest", dict(kT=args.kT, storage=BF16), 108),
                ("aa_reg_flbm", (e, e, e), "rest", dict(kT=args.kT, storage=F32, pattern=AA), 216),
                ("aa_reg_lbm_kT0", (e, e, e), "rest", dict(kT=0.0, storage=F32, pattern=AA), 216),
                ("aa_f16_reg_flbm", (e, e, e), "rest", dict(kT=args.kT, storage=F16, pattern=AA), 108),
                # mixed precision at 512^3 (134 M sites), float32 beside it on the same GPU
                ("c3_512_f32_reg_flbm", (512,) * 3, "rest", dict(kT=1e-4, storage=F32), 216),
                ("c3_512_f16_reg_flbm", (512,) * 3, "rest", dict(kT=1e-4, storage=F16), 108),
                ("c3_512_bf16_reg_flbm", (512,) * 3, "rest", dict(kT=1e-4, storage=BF16), 108),
                # large single boxes from the Taylor-Green vortex (u0 0.01) with noise
                ("c5_768_f32_reg_flbm", (768,) * 3, "taylor-green", dict(kT=1e-4, storage=F32), 216),
                ("c5_1024_f16_aa_reg_flbm", (1024,) * 3, "taylor-green",
                 dict(kT=1e-4, storage=F16, pattern=AA), 108)):
            variants[name] = time_variant(R, torch, stream, shape, k, peak_v, bps, init=init,
                                          kernel=kernel, **kw)
        accuracy = storage_accuracy(R, torch, stream)
        # batched ensemble: 64 replicas of uneven sizes, one CUDA graph of per-step launches per call
        from paper_2507_08820_gb300 import workloads as W
        reps = W.replica_ensemble(64, seed=0)
        sites = sum(r["nx"] * r["ny"] * r["nz"] for r in reps)
        for name, st_b, bps in (("batch64_f32", R.RFLBM_STORE_F32, 216),
                                ("batch64_f16", R.RFLBM_STORE_F16, 108)):
            bh = R.rflbm_batch_create(reps, storage=st_b, tile=0)
            R.rflbm_batch_init_rest(bh)
            R.rflbm_batch_run(bh, 20)
            k = max(200, args.steps // 20)
            R.rflbm_batch_prepare(bh, k)
            R.rflbm_batch_synchronize(bh)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(torch.cuda.default_stream())
            R.rflbm_batch_run(bh, k)
            ev1.record(torch.cuda.default_stream())
            ev1.synchronize()
            sites_s = sites * k / (ev0.elapsed_time(ev1) * 1e-3)
            tile, per_sm, _ = R.rflbm_batch_tuning(bh)
            variants[name] = {"value": sites_s / 1e6, "unit": "MLUPS", "steps": k,
                              "replicas": len(reps), "sites": sites, "tile": "autotuned per row length",
                              "roofline_frac": bps * sites_s / 1e9 / peak_v, "bytes_per_site": bps}
            R.rflbm_batch_destroy(bh)
    box.close()

    if info.rank != 0:
        dist.finalize(info)
        return 0
    value = info.world * n * args.steps / (ms_max * 1e-3) / 1e6
    per_launch_s = ms * 1e-3 / args.steps
    achieved = BYTES_PER_SITE[args.storage] * n / per_launch_s / 1e9
    peak, peak_kind = measured_peak()
    kname, kstem = kernel_name(kind, path, args.kT, 0, args.storage, args.pattern, pairs, odd_pairs)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None if slab else profiled_traffic(kstem, e),
                "peak_source": f"hbm_gbs of {peak_kind}", "kernel": kname,
                "algorithmic_bytes_per_launch": BYTES_PER_SITE[args.storage] * n}
    rings = None
    if slab:
        roofline["kernel"] = f"{kname}: boundary rows, interior rows, face exchange (per step)"
        roofline["algorithmic_bytes_per_step"] = roofline.pop("algorithmic_bytes_per_launch")
        if info.world == 1:
            rings = slab_rings(R, torch, args, peak)
    cpu = None
    if not args.no_cpu_baseline and info.world == 1:  # the oracle baseline is an N = 1 figure
        r = oracle_sample_rate(e, args.tau, args.kT, budget_s=12.0, steps=None)
        cpu = cpu_baseline_entry(r, e, False)
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": info.world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "storage_dtype": args.storage, "data": "synthetic", "config": workload(args, info.world),
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
        "stats_after": {"mass_rel_drift": (st.mass - n) / n, "max_speed": st.max_speed,
                        "nonfinite": st.nonfinite},
        "variants": variants,
        "storage_accuracy": accuracy,
    }
    if rings is not None:
        line["slab_rings_one_gpu"] = rings
    print(json.dumps(line))
    dist.finalize(info)
    return 0


def backtransform_arm(args):
    """The back transform of Eq. 11 on its own: float32 FMAs (as in the step kernels) against
    tcgen05 MMA over tiles of 128 sites with split-bfloat16 moments. Each site transforms
    `reps` sets of moments held in registers, so no population crosses DRAM. Also the noise
    draw of a step on its own (24 normals per site), the bound of the 16-bit steps."""
    from paper_2507_08820_gb300 import build
    build.build()
    from paper_2507_08820_gb300 import rflbm as R
    tiles, reps = 152 * 32, 64
    out = {"metric": "Eq. 11 back transforms per second, float32 FMA vs tcgen05 MMA", "unit": "G site transforms/s",
           "workload": f"{tiles} tiles of 128 sites x {reps} transforms each, moments in registers",
           "higher_is_better": True}
    for name, method in (("fma", 0), ("mma", 1)):
        R.rflbm_testing_backtransform_time(method, tiles, reps)
        ms = min(R.rflbm_testing_backtransform_time(method, tiles, reps) for _ in range(3))
        out[name] = {"ms": ms, "value": tiles * 128 * reps / (ms * 1e-3) / 1e9}
    # the forward projection (the ten moments of order <= 2) alone, FMA vs float16 MMA
    out["forward"] = {"workload": f"{tiles} tiles of 128 sites x {reps} projections each, float16 populations "
                                  "in registers", "unit": "G site projections/s"}
    for name, method in (("fma", 0), ("mma", 1)):
        R.rflbm_testing_forward_time(method, tiles, reps)
        ms = min(R.rflbm_testing_forward_time(method, tiles, reps) for _ in range(3))
        out["forward"][name] = {"ms": ms, "value": tiles * 128 * reps / (ms * 1e-3) / 1e9}
    # the noise draw of a step alone, against the sites per second of the 16-bit roofline
    nsites = 1 << 27
    R.rflbm_testing_noise_time(nsites)
    ms = min(R.rflbm_testing_noise_time(nsites) for _ in range(3))
    peak, kind = measured_peak()
    rate = nsites / (ms * 1e-3)
    out["noise_draw_alone"] = {"ms": ms, "sites": nsites, "value": rate / 1e9, "unit": "G sites/s",
                               "fraction_of_16bit_roofline": rate * 108 / 1e9 / peak,
                               "peak": f"hbm_gbs of {kind}"}
    print(json.dumps(out))
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    if args.workload == "ensemble":
        return ensemble_arm(args)
    if args.workload == "backtransform":
        return backtransform_arm(args)
    return gb300_arm(args)


if __name__ == "__main__":
    sys.exit(main())
