"""Benchmark of the FDTD + CPML hot path on GB300.

Workload (one bench "step"): the 512^3 layered-model run — 10 layers
1500-4500 m/s (seed 2), dx = 10 m, CFL 0.5, 20 CPML cells per face,
R = 1e-8, 10 Hz Ricker 30 cells below the top face — advanced 1000 time steps
from a zero state.  Metric: million output points per second,
N^3 * Nt / (1e6 T) (paper Sec. 5), and the fraction of the measured HBM
bandwidth reached by the step kernel.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--storage f32|f16|bf16]
                    [--impl ours|reference] [--nt 1000] [--no-cpu-baseline]

Multi-GPU: replicas only (the grid is not decomposed; each rank runs its own
copy of the workload), launched by torch.distributed.run; rank 0 prints the
JSON line with the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "million output points/s and % of HBM peak, plain FP32 vs chosen forms"
UNIT = "Mpoints/s"


def cells_arg(text: str):
    v = [int(x) for x in text.split(",")]
    if len(v) == 1:
        v = v * 6
    if len(v) != 6 or min(v) < 0:
        raise argparse.ArgumentTypeError("one count or six counts >= 0")
    return tuple(v)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16"])
    ap.add_argument("--preset", default="layered512")
    ap.add_argument("--nt", type=int, default=None, help="time steps per bench step (default: the workload's)")
    ap.add_argument("--cells", type=cells_arg, default=None,
                    help="override CPML cells: one count for every face (0: no CPML), or six comma-separated "
                         "counts -x,+x,-y,+y,-z,+z (profiling runs of one axis' layer)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-accuracy", dest="accuracy", action="store_false",
                    help="skip the 128^3 accuracy instance of the cpu_baseline leg")
    ap.add_argument("--forms-only", action="store_true", help="measure only the forms (profiling runs)")
    ap.add_argument("--variant", default="plain", choices=["plain", "staggered", "local", "density"],
                    help="form of the main line's step (profiling runs of the forms; FP32): the staggered grid "
                         "at CFL 0.4, the local-velocity CPML grading, or the density (c/1500)^(1/4)")
    ap.add_argument("--oracle-sample", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--forms", default="f16,bf16,cpml_overhead,adjoint,learned,tblock,decomp,density,aniso2d,staggered,local_cpml",
                    help="comma list of forms measured after the main line ('' for none)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(ms: float, dist, device) -> float:
    """The slowest rank's time (every rank gets it); `dist` is None on one rank."""
    if dist is None:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world: int, npts: float, nt: int, steps: int, total_ms: float) -> float:
    """Mpoints/s of the whole job: every rank advances its own replica of the
    grid (weak scaling), all in the slowest rank's time."""
    return world * npts * nt * steps / (total_ms * 1e-3) / 1e6


# ----------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        # the raw samples: a temporary folder unless FDTD_CLOCKS_DIR names one
        out_dir = os.environ.get("FDTD_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"fdtd_clocks_rank{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
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
        self.f.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def step_kernel_source_hash() -> str:
    """Hash of what decides a step kernel launch: its device code (fdtd_step.cu
    and the shared declarations of fdtd_internal.cuh up to the host-only
    context struct) and the host code that sets its launch (fdtd_api.cu: the
    z-chunking, the tile order's columns, the arguments)."""
    csrc = os.path.join(ROOT, "paper_2606_06910_gb300", "csrc")
    step = open(os.path.join(csrc, "fdtd_step.cu"), "rb").read()
    inc = open(os.path.join(csrc, "fdtd_internal.cuh"), "rb").read()
    api = open(os.path.join(csrc, "fdtd_api.cu"), "rb").read()
    cut = inc.find(b"// The opaque context behind fdtd_ctx*.")
    return hashlib.sha256(step + (inc[:cut] if cut >= 0 else inc) + api).hexdigest()[:16]


def step_kernel_traffic(storage: str, shape, variant: str = "plain"):
    """DRAM bytes per launch of the step kernel from the committed ncu summary,
    scaled to this grid, or None when the kernel source changed since (forms
    other than the plain one are keyed "<storage>-<variant>")."""
    path = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    h = step_kernel_source_hash()
    e = d.get(storage if variant == "plain" else f"{storage}-{variant}")
    if not e or e.get("kernel_sha") != h:
        return None
    n_prof = float(np.prod(e["shape"]))
    return float(e["dram_bytes_per_launch"]) * float(np.prod(shape)) / n_prof


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
def algorithmic_bytes(shape, cells, es, variant="plain"):
    """Per launch: read p, v (3), K and write p, v (3): 8 stored words + one
    FP32 word per node; plus 4 stored words (psi_v and psi_p read and write)
    per slab node and axis.  The density form reads one more FP32 word per
    node (dt / rho); the local grading reads b and a (8 B) per slab node and
    axis; the staggered form moves the same bytes."""
    nz, ny, nx = shape
    n = nx * ny * nz
    slab = (cells[0] + cells[1]) * ny * nz + (cells[2] + cells[3]) * nx * nz + (cells[4] + cells[5]) * nx * ny
    extra = 4 * n if variant == "density" else (8 * slab if variant == "local" else 0)
    return (8 * es + 4) * n + 4 * es * slab + extra


def run_ours(args, rank, world, local):
    import torch
    from paper_2606_06910_gb300 import synth
    from paper_2606_06910_gb300.fdtd import Fdtd

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    w = synth.preset(args.preset)
    nt = args.nt or w.nt
    cells = w.cpml_cells if args.cells is None else args.cells
    shape = w.shape
    vel_h = w.velocity()
    src = w.sources()
    variant = args.variant
    if variant != "plain" and args.storage != "f32":
        raise SystemExit("--variant needs --storage f32")
    dt = 0.4 * w.h / w.c_max if variant == "staggered" else w.dt     # the staggered limit is 0.4488
    wav_h = synth.ricker(nt, dt, w.f0).astype(np.float32)[None, :]
    stream = torch.cuda.current_stream(dev)

    sim = Fdtd(shape, w.h, dt, cpml_cells=cells, storage=args.storage, nt_max=nt, device=dev, stream=stream,
               cpml_local=variant == "local")
    vel = torch.from_numpy(vel_h).to(dev)
    wav = torch.from_numpy(wav_h).to(dev)
    if variant == "staggered":
        sim.set_staggered(True)
    sim.set_model(vel, (vel / 1500.0) ** 0.25 if variant == "density" else None)
    if any(cells):
        if variant == "local":
            sim.set_cpml_local(vel, R=w.R, kappa_max=w.kappa_max, alpha_frac=w.alpha_frac, q=w.q)
        else:
            sim.set_cpml(R=w.R, kappa_max=w.kappa_max, alpha_frac=w.alpha_frac, q=w.q, c_ref=w.c_max)
    sim.inject(src, wav)

    def one_step(evs=None):
        sim.reset()
        if evs is not None:
            evs[0].record(stream)
        sim.step(nt)
        if evs is not None:
            evs[1].record(stream)

    for _ in range(args.warmup):
        one_step()
    sim.sync()

    dist = None
    if world > 1:
        import torch.distributed as dist
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t0.record(stream)
    for k in range(args.steps):
        one_step(kev[k])
    t1.record(stream)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    clk = clocks.stop()
    sim.sync()
    total_ms = t0.elapsed_time(t1)
    kernel_ms = sum(a.elapsed_time(b) for a, b in kev)
    total_ms = max_over_ranks(total_ms, dist, dev)
    npts = float(np.prod(shape))
    value = whole_job_value(world, npts, nt, args.steps, total_ms)

    # roofline of the step kernel (the only kernel of sim.step)
    es = 4 if args.storage == "f32" else 2
    launches = args.steps * nt
    avg_launch_s = kernel_ms * 1e-3 / launches
    bytes_launch = algorithmic_bytes(shape, cells, es, variant)
    achieved = bytes_launch / avg_launch_s / 1e9
    peak, peak_kind = measured_peaks()
    traffic = step_kernel_traffic(args.storage, shape, variant)

    # end to end through the public API: every step copies its model and
    # wavelet in from pinned host memory and its pressure snapshot out to
    # pinned host memory.  The copies run on a stream of their own, double
    # buffered: step k+1's inputs go up and step k-1's snapshot comes down
    # while step k computes; the timed region ends when the last snapshot is
    # on the host.
    e2e = None
    if not args.no_e2e and variant == "plain":
        vel_pin = torch.from_numpy(vel_h).pin_memory()
        wav_pin = torch.from_numpy(wav_h).pin_memory()
        snap_pin = [torch.empty(shape, dtype=torch.float32).pin_memory() for _ in range(2)]
        vel_d = [torch.empty_like(vel) for _ in range(2)]
        wav_d = [torch.empty_like(wav) for _ in range(2)]
        snap_d = [torch.empty(shape, dtype=torch.float32, device=dev) for _ in range(2)]
        copy = torch.cuda.Stream(dev)
        ksteps = args.steps
        up = [torch.cuda.Event() for _ in range(2)]
        done = [torch.cuda.Event() for _ in range(2)]
        down = [torch.cuda.Event() for _ in range(2)]

        def upload(k):
            b = k % 2
            with torch.cuda.stream(copy):
                copy.wait_event(done[b])          # step k-2 no longer reads buffer b
                vel_d[b].copy_(vel_pin, non_blocking=True)
                wav_d[b].copy_(wav_pin, non_blocking=True)
                up[b].record(copy)

        def download(k):
            b = k % 2
            with torch.cuda.stream(copy):
                copy.wait_event(done[b])          # step k's snapshot is in buffer b
                snap_pin[b].copy_(snap_d[b], non_blocking=True)
                down[b].record(copy)

        torch.cuda.synchronize(dev)
        e0 = time.perf_counter()
        upload(0)
        for k in range(ksteps):
            b = k % 2
            stream.wait_event(up[b])
            stream.wait_event(down[b])            # snapshot k-2 has left buffer b
            sim.set_model(vel_d[b])               # synchronises the compute stream
            # the previous snapshot goes down, and the next inputs go up, while
            # this step computes; issued after set_model, whose small read-back
            # then does not queue behind a large copy
            if k >= 1:
                download(k - 1)
            if k + 1 < ksteps:
                upload(k + 1)
            sim.inject(src, wav_d[b])
            sim.reset()
            sim.step(nt)
            sim.get("p", 0, snap_d[b])
            done[b].record(stream)
        download(ksteps - 1)
        torch.cuda.synchronize(dev)
        e_s = time.perf_counter() - e0
        e2e = {"value": round(world * npts * nt * ksteps / e_s / 1e6, 2), "unit": UNIT,
               "h2d_bytes_per_step": int(vel_pin.numel() * 4 + wav_pin.numel() * 4 + src.size * 4),
               "d2h_bytes_per_step": int(snap_pin[0].numel() * 4),
               "copies": "on their own stream, double buffered, overlapping the neighbouring steps"}
    sim.sync()
    out = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.storage, "data": "synthetic",
        "config": workload_config(args, shape, cells, nt, world),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": None if traffic is None else round(traffic),
                     "peak_source": f"{peak_kind} hbm_gbs", "kernel": "fdtd_step_kernel",
                     "algorithmic_bytes_per_launch": int(bytes_launch),
                     "avg_launch_us": round(avg_launch_s * 1e6, 2)},
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
    }
    return out


# ----------------------------------------------------------------------------
# the forms measured next to the FP32 path
# ----------------------------------------------------------------------------
def _timed(stream, fn):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) * 1e-3


def form_storage(storage, dev, nsteps=60, warm=10):
    """16-bit storage on the 1024^3 layered workload (20 CPML cells)."""
    import torch
    from paper_2606_06910_gb300 import synth
    from paper_2606_06910_gb300.fdtd import Fdtd
    w = synth.preset("layered1024")
    sim = Fdtd(w.shape, w.h, w.dt, cpml_cells=w.cpml_cells, storage=storage, nt_max=w.nt, device=dev)
    sim.set_model(torch.from_numpy(w.velocity()).to(dev))
    sim.set_cpml(R=w.R, c_ref=w.vmax)
    sim.inject(w.sources(), torch.from_numpy(w.wavelet()).to(dev))
    sim.step(warm)
    sim.sync()
    secs = _timed(sim.stream, lambda: sim.step(nsteps))
    sim.sync()
    npts = float(np.prod(w.shape))
    bytes_launch = algorithmic_bytes(w.shape, w.cpml_cells, 2)
    peak, kind = measured_peaks()
    del sim
    torch.cuda.empty_cache()
    ach = bytes_launch * nsteps / secs / 1e9
    return {"workload": f"layered1024 {storage} storage, {nsteps} timed steps", "value": round(npts * nsteps / secs / 1e6, 1),
            "unit": UNIT, "roofline_frac": round(ach / peak, 4), "achieved_GBps": round(ach, 1)}


ACCURACY_CHECKPOINTS = (250, 375, 500)


def storage_accuracy_gpu(dev, storage):
    """The precision form's 128^3 accuracy instance (same generator as the
    1024^3 workload, seed 3, 500 steps) on the GPU: the pressure after steps
    250, 375 and 500 and the receiver traces, as host arrays."""
    import torch
    from paper_2606_06910_gb300 import synth
    from paper_2606_06910_gb300.fdtd import Fdtd
    w = synth.preset("layered128")
    rec = synth.receiver_grid(w.shape, w.cpml_cells, 6, 6, w.cpml_cells[4])
    sim = Fdtd(w.shape, w.h, w.dt, cpml_cells=w.cpml_cells, storage=storage, nt_max=w.nt, nrec_max=len(rec),
               device=dev)
    sim.set_model(torch.from_numpy(w.velocity()).to(dev))
    sim.set_cpml(R=w.R, c_ref=w.vmax)
    sim.inject(w.sources(), torch.from_numpy(w.wavelet()).to(dev))
    traces = sim.record(rec)
    out, t = {}, 0
    for c in ACCURACY_CHECKPOINTS:
        sim.step(c - t)
        t = c
        out[c] = sim.get("p").cpu().numpy().astype(np.float64)
    sim.sync()
    out["traces"] = traces[0].cpu().numpy().astype(np.float64)
    sim.close()
    return out


def form_cpml_overhead(dev, nsteps=96, warm=8):
    """CPML overhead as the paper defines it (Sec. 5): (T_CPML - T_none) /
    T_none, on the 512^3 layered workload with 20 cells per face and with
    none, same grid, source and steps; both times are the step kernel's own
    launch times from the library's CUDA events."""
    import torch
    from paper_2606_06910_gb300 import synth
    from paper_2606_06910_gb300.fdtd import Fdtd
    w = synth.preset("layered512")
    vel = torch.from_numpy(w.velocity()).to(dev)
    npts = float(np.prod(w.shape))
    peak, _ = measured_peaks()
    out = {}
    for name, cells in (("cpml_20", w.cpml_cells), ("none", (0,) * 6)):
        sim = Fdtd(w.shape, w.h, w.dt, cpml_cells=cells, nt_max=w.nt, device=dev)
        sim.set_model(vel)
        if any(cells):
            sim.set_cpml(R=w.R, c_ref=w.vmax)
        sim.inject(w.sources(), torch.from_numpy(w.wavelet()).to(dev))
        sim.step(warm)
        sim.sync()
        sim.set_timing(True)
        secs = _timed(sim.stream, lambda: sim.step(nsteps))
        kms, nl = sim.timing("step")
        b = algorithmic_bytes(w.shape, cells, 4)
        out[name] = {"value": round(npts * nsteps / secs / 1e6, 1), "ms_per_step": round(secs / nsteps * 1e3, 4),
                     "kernel_ms_per_launch": round(kms / nl, 4),
                     "roofline_frac": round(b / (kms / nl * 1e-3) / 1e9 / peak, 4)}
        del sim
        torch.cuda.empty_cache()
    t1, t0 = out["cpml_20"]["kernel_ms_per_launch"], out["none"]["kernel_ms_per_launch"]
    b1 = algorithmic_bytes(w.shape, w.cpml_cells, 4)
    b0 = algorithmic_bytes(w.shape, (0,) * 6, 4)
    return {"workload": f"layered512, 20 CPML cells vs none, {warm} + {nsteps} timed steps", "unit": UNIT, **out,
            "overhead": round((t1 - t0) / t0, 4),
            "byte_floor": round((b1 - b0) / b0, 4),
            "target": 0.03}


def form_decomp(dev, nsteps=48, warm=8):
    """The paper's pencil-yz decomposition (Sec. 3.3) on one GPU: the 512^3
    layered workload split into 1 x 2 x 2 parts with ghosts of depth 8 s,
    exchanged every s steps (s = 1, 2, 4), against the undivided grid.
    The parts run on streams of their own, side by side.  Reports ms per
    step, the time of one exchange phase (timed alone, every part's ghosts
    refreshed), the redundant ghost work, and whether the assembled pressure
    equals the undivided grid's bit for bit."""
    import torch
    from paper_2606_06910_gb300 import synth
    from paper_2606_06910_gb300.decomp import Decomposition
    from paper_2606_06910_gb300.fdtd import Fdtd
    w = synth.preset("layered512")
    vel = torch.from_numpy(w.velocity()).to(dev)
    npts = float(np.prod(w.shape))
    out = {}
    sim = Fdtd(w.shape, w.h, w.dt, cpml_cells=w.cpml_cells, nt_max=w.nt, device=dev)
    sim.set_model(vel)
    sim.set_cpml(R=w.R, c_ref=w.vmax)
    sim.inject(w.sources(), torch.from_numpy(w.wavelet()).to(dev))
    sim.step(warm)
    secs = _timed(sim.stream, lambda: sim.step(nsteps))
    p_ref = sim.get("p").clone()
    out["single"] = {"value": round(npts * nsteps / secs / 1e6, 1), "ms_per_step": round(secs / nsteps * 1e3, 4)}
    sim.close()
    del sim
    torch.cuda.empty_cache()
    for s in (1, 2, 4):
        dec = Decomposition(w.shape, w.h, w.dt, parts=(1, 2, 2), s=s, cpml_cells=w.cpml_cells, nt_max=w.nt, device=dev)
        dec.set_model(vel)
        dec.set_cpml(R=w.R, c_ref=w.vmax)
        dec.inject(w.sources(), torch.from_numpy(w.wavelet()).to(dev))
        dec.step(warm)
        dec.sync()
        secs = _timed(dec.stream, lambda: dec.step(nsteps))
        same = bool(torch.equal(dec.get("p"), p_ref))

        def exchanges(k=16):
            # the exchange phase alone (ordered as in a step block)
            dec._parts_wait_main()
            for _ in range(k):
                dec._barrier()
                dec.exchange()
                dec._barrier()
            dec._main_waits_parts()
        ex_s = _timed(dec.stream, exchanges) / 16
        local = sum(float(np.prod([hi - lo for lo, hi in sub["loc"]])) for sub in dec.subs)
        out[f"s{s}"] = {"value": round(npts * nsteps / secs / 1e6, 1), "ms_per_step": round(secs / nsteps * 1e3, 4),
                        "exchange_ms_per_exchange": round(ex_s * 1e3, 4),
                        "exchange_ms_per_step": round(ex_s / s * 1e3, 4), "ghost_depth": 8 * s,
                        "computed_over_owned_nodes": round(local / npts, 4), "identical_to_single": same}
        dec.close()
        del dec
        torch.cuda.empty_cache()
    return {"workload": f"layered512 pencil-yz 1x2x2 parts on one GPU, {warm} + {nsteps} timed steps", "unit": UNIT,
            **out}


def form_tblock(dev, nsteps=96, warm=8):
    """Temporal blocking sweep k = 1, 2, 4 on the 512^3 layered workload
    (20 CPML cells): Mpoints/s of each k, and whether the final state of k = 2
    and 4 equals the one of k = 1 node for node."""
    import torch
    from paper_2606_06910_gb300 import synth
    from paper_2606_06910_gb300.fdtd import Fdtd
    w = synth.preset("layered512")
    npts = float(np.prod(w.shape))
    out, p_ref = {}, None
    for k in (1, 2, 4):
        sim = Fdtd(w.shape, w.h, w.dt, cpml_cells=w.cpml_cells, nt_max=w.nt, tblock_k=k, device=dev)
        sim.set_model(torch.from_numpy(w.velocity()).to(dev))
        sim.set_cpml(R=w.R, c_ref=w.vmax)
        sim.inject(w.sources(), torch.from_numpy(w.wavelet()).to(dev))
        sim.step(warm)
        sim.sync()
        secs = _timed(sim.stream, lambda: sim.step(nsteps))
        sim.sync()
        p = sim.get("p")
        entry = {"value": round(npts * nsteps / secs / 1e6, 1), "ms_per_step": round(secs / nsteps * 1e3, 4)}
        if p_ref is None:
            p_ref = p.clone()
        else:
            entry["identical_to_k1"] = bool(torch.equal(p, p_ref))
        out[f"k{k}"] = entry
        del sim, p
        torch.cuda.empty_cache()
    return {"workload": f"layered512, {warm} + {nsteps} timed steps, z bands of 96 planes in 32-plane chunks",
            "unit": UNIT, **out}


def form_density(dev, nsteps=96, warm=8):
    """Variable density on the 512^3 layered workload: density (c / 1500)^(1/4)
    per node (a Gardner-type relation, dimensionless), against the same run
    with density 1; Mpoints/s of both."""
    import torch
    from paper_2606_06910_gb300 import synth
    from paper_2606_06910_gb300.fdtd import Fdtd
    w = synth.preset("layered512")
    vel = torch.from_numpy(w.velocity()).to(dev)
    rho = (vel / 1500.0) ** 0.25
    npts = float(np.prod(w.shape))
    out = {}
    peak, _ = measured_peaks()
    for name, r in (("constant", None), ("variable", rho)):
        sim = Fdtd(w.shape, w.h, w.dt, cpml_cells=w.cpml_cells, nt_max=w.nt, device=dev)
        sim.set_model(vel, r)
        sim.set_cpml(R=w.R, c_ref=w.vmax)
        sim.inject(w.sources(), torch.from_numpy(w.wavelet()).to(dev))
        sim.step(warm)
        sim.sync()
        secs = _timed(sim.stream, lambda: sim.step(nsteps))
        b = algorithmic_bytes(w.shape, w.cpml_cells, 4, "density" if r is not None else "plain")
        out[name] = {"value": round(npts * nsteps / secs / 1e6, 1), "ms_per_step": round(secs / nsteps * 1e3, 4),
                     "roofline_frac": round(b * nsteps / secs / 1e9 / peak, 4)}
        del sim
        torch.cuda.empty_cache()
    return {"workload": f"layered512, density (c/1500)^0.25, {warm} + {nsteps} timed steps", "unit": UNIT, **out}


def form_staggered(dev, nsteps=96, warm=8):
    """The staggered (Yee) form on the 512^3 layered workload (20 CPML cells)
    at CFL 0.4 (its limit is 0.4488), against the collocated form at the same
    dt: Mpoints/s and the fraction of measured HBM bandwidth of each (the
    same algorithmic bytes per step)."""
    import torch
    from paper_2606_06910_gb300 import synth
    from paper_2606_06910_gb300.fdtd import Fdtd
    w = synth.preset("layered512")
    dt = 0.4 * w.h / w.vmax
    vel = torch.from_numpy(w.velocity()).to(dev)
    npts = float(np.prod(w.shape))
    bytes_launch = algorithmic_bytes(w.shape, w.cpml_cells, 4)
    peak, _ = measured_peaks()
    out = {}
    for name in ("collocated", "staggered"):
        sim = Fdtd(w.shape, w.h, dt, cpml_cells=w.cpml_cells, nt_max=w.nt, device=dev)
        sim.set_staggered(name == "staggered")
        sim.set_model(vel)
        sim.set_cpml(R=w.R, c_ref=w.vmax)
        sim.inject(w.sources(), torch.from_numpy(w.wavelet()).to(dev))
        sim.step(warm)
        sim.sync()
        secs = _timed(sim.stream, lambda: sim.step(nsteps))
        ach = bytes_launch * nsteps / secs / 1e9
        out[name] = {"value": round(npts * nsteps / secs / 1e6, 1), "ms_per_step": round(secs / nsteps * 1e3, 4),
                     "roofline_frac": round(ach / peak, 4)}
        del sim
        torch.cuda.empty_cache()
    return {"workload": f"layered512 at CFL 0.4, {warm} + {nsteps} timed steps", "unit": UNIT, **out}


def form_local_cpml(dev, nsteps=96, warm=8):
    """Local-velocity CPML grading on the 512^3 layered workload (20 cells):
    b, a per slab node from the node's velocity, against the 1D grading with
    c_ref = c_max; Mpoints/s of both.  The per-node tables add 8 B per slab
    node and axis read per step."""
    import torch
    from paper_2606_06910_gb300 import synth
    from paper_2606_06910_gb300.fdtd import Fdtd
    w = synth.preset("layered512")
    vel = torch.from_numpy(w.velocity()).to(dev)
    npts = float(np.prod(w.shape))
    out = {}
    peak, _ = measured_peaks()
    for name in ("1d", "local"):
        sim = Fdtd(w.shape, w.h, w.dt, cpml_cells=w.cpml_cells, nt_max=w.nt, cpml_local=name == "local", device=dev)
        sim.set_model(vel)
        if name == "local":
            sim.set_cpml_local(vel, R=w.R)
        else:
            sim.set_cpml(R=w.R, c_ref=w.vmax)
        sim.inject(w.sources(), torch.from_numpy(w.wavelet()).to(dev))
        sim.step(warm)
        sim.sync()
        secs = _timed(sim.stream, lambda: sim.step(nsteps))
        b = algorithmic_bytes(w.shape, w.cpml_cells, 4, "local" if name == "local" else "plain")
        out[name] = {"value": round(npts * nsteps / secs / 1e6, 1), "ms_per_step": round(secs / nsteps * 1e3, 4),
                     "roofline_frac": round(b * nsteps / secs / 1e9 / peak, 4)}
        del sim
        torch.cuda.empty_cache()
    return {"workload": f"layered512, {warm} + {nsteps} timed steps", "unit": UNIT, **out}


def form_aniso2d(dev, nt=1000, every=50):
    """The paper's 2D anisotropic CPML demonstration (Sec. 5): sum p^2 inside
    the layer relative to its peak, with a 10-cell layer and with none."""
    from paper_2606_06910_gb300 import demos
    t0 = time.perf_counter()
    _, e_c, cfg, _ = demos.anisotropic_2d(True, nt, every, device=dev)
    secs = time.perf_counter() - t0
    _, e_n, _, _ = demos.anisotropic_2d(False, nt, every, device=dev)
    dt = cfg["dt"]
    curve = {f"{(k + 1) * every * dt:.3f}s": [float(f"{e_c[k] / e_c.max():.3e}"), float(f"{e_n[k] / e_n.max():.3e}")]
             for k in range(0, len(e_c), 4)}
    return {"workload": f"2 km x 2 km, 8 m, c_x 2600 / c_z 1800 m/s, 30 Hz, {nt} steps",
            "final_over_peak_cpml": float(f"{e_c[-1] / e_c.max():.3e}"),
            "final_over_peak_no_cpml": float(f"{e_n[-1] / e_n.max():.3e}"),
            "curve_cpml_vs_none": curve, "wall_s_cpml_run": round(secs, 3)}


def form_adjoint(dev, nt=800, nshots=None, every=None):
    """Forward with checkpoints + discrete adjoint, 256^3 x 16 shots, 128x128
    receivers, checkpoint every 50 steps (gradient of the L2 misfit).  The form
    spec "adjoint:S:N" runs S shots over N steps with a checkpoint every N
    (the small case the profiles use)."""
    import torch
    from paper_2606_06910_gb300 import synth
    from paper_2606_06910_gb300.fdtd import Fdtd
    w = synth.preset("adjoint256")
    rec = synth.receiver_grid(w.shape, w.cpml_cells, *w.extra["receivers"], z=w.cpml_cells[4])
    c0 = synth.gaussian_smooth(w.velocity(), w.extra["smooth_sigma"])
    ns = w.nshots if nshots is None else nshots
    every = w.extra["checkpoint_every"] if every is None else every
    sim = Fdtd(w.shape, w.h, w.dt, nshots=ns, cpml_cells=w.cpml_cells, nt_max=nt, nrec_max=len(rec),
               checkpoint_every=every, device=dev)
    sim.set_model(torch.from_numpy(c0).to(dev))
    sim.set_cpml(R=w.R, c_ref=w.vmax)
    sim.inject(w.sources()[:ns], torch.from_numpy(w.wavelet(nt)[:ns]).to(dev))
    sim.record(rec)
    dobs = torch.zeros_like(sim.traces)
    grad = torch.zeros(w.shape, device=dev)
    resid = torch.empty_like(sim.traces)
    t_fwd = _timed(sim.stream, lambda: sim.step(nt))
    J = sim.misfit(dobs, nt=nt, resid=resid)
    sim.set_timing(True)
    t_adj = _timed(sim.stream, lambda: sim.adjoint(nt, resid, grad))
    adj_ms, adj_n = sim.timing("adjoint")
    rec_ms, rec_n = sim.timing("step")
    sim.sync()
    ok = bool(torch.isfinite(grad).all()) and float(grad.abs().max()) > 0
    pts = float(np.prod(w.shape)) * ns * nt
    # fused adjoint kernel: read mu, lam_v (3), kdt, the taped bracket and
    # dJ/dK, write mu, lam_v (3) and dJ/dK: 12 FP32 words per node and shot;
    # plus the adjoint memory variables (read + write of two) per slab node
    # and axis
    nz, ny, nx = w.shape
    cl = w.cpml_cells
    slab = (cl[0] + cl[1]) * ny * nz + (cl[2] + cl[3]) * nx * nz + (cl[4] + cl[5]) * nx * ny
    adj_bytes = ns * (48 * float(np.prod(w.shape)) + 16 * slab)
    peak, kind = measured_peaks()
    per_launch = adj_ms / max(adj_n, 1) * 1e-3
    ach = adj_bytes / per_launch / 1e9
    del sim
    torch.cuda.empty_cache()
    return {"workload": f"adjoint256: 256^3 x {ns} shots x {nt} steps, C={every}", "value": round(pts / (t_fwd + t_adj) / 1e6, 1),
            "unit": UNIT + " (forward + adjoint)", "forward_s": round(t_fwd, 3), "adjoint_s": round(t_adj, 3),
            "misfit": J, "gradient_finite_nonzero": ok,
            "recompute_step_launches": rec_n, "recompute_ms_per_launch": round(rec_ms / max(rec_n, 1), 4),
            "roofline": {"bound": "hbm", "kernel": "adj_fused_kernel", "launches": adj_n,
                         "avg_launch_us": round(per_launch * 1e6, 2), "algorithmic_bytes_per_launch": int(adj_bytes),
                         "achieved": round(ach, 1), "peak": peak, "unit": "GB/s", "frac": round(ach / peak, 4),
                         "peak_source": f"{kind} hbm_gbs"}}


def form_learned(dev, iters=48, eval_freqs=(12.0, 20.0)):
    """Learned 6-cell CPML: trained through the adjoint on 96^3 homogeneous
    reflection runs (c = 2000 m/s; four frequency groups drawn from 5-30 Hz;
    sources meeting seeded faces at seeded angles 0-80 degrees), evaluated on
    the 512^3 layered model (seed 5, 1000 steps) at two frequencies inside the
    training range, against the polynomial grading with 6 and 20 cells:
    reflection ratio ||traces - reference|| / ||reference|| at receivers just
    inside the layer, the reference being the same interior inside a grid 64
    nodes larger per side.  The network is asked for the evaluation's
    reference velocity (c_max = 4500 m/s), time step and frequency."""
    import torch
    from paper_2606_06910_gb300 import synth
    from paper_2606_06910_gb300.fdtd import Fdtd
    from paper_2606_06910_gb300.learned import misfit_flat, reflection_task, train_learned_cpml
    t0 = time.perf_counter()
    task = reflection_task(n=96, L=6, nshots=8, seed=3, freqs=(5.0, 30.0), nfreq=4, angles=(0.0, 80.0), device=dev)
    res = train_learned_cpml(task, iters=iters, lr=5e-3, seed=0)
    t_train = time.perf_counter() - t0
    model = res["model"]
    n, nt, h, margin, cmax = 512, 1000, 10.0, 64, 4500.0
    vel = synth.layered_model((n,) * 3, seed=5)
    dt = 0.5 * h / cmax
    src = np.array([[n // 2, n // 2 + 37, n // 2 - 51]], np.int32)
    rec = synth.face_receivers(n, 20, 8, inset=6)
    nb = n + 2 * margin
    vb = np.pad(vel, margin, mode="edge")
    evals = {}
    for f0 in eval_freqs:
        wav = synth.ricker(nt, dt, f0).astype(np.float32)[None, :]
        big = Fdtd((nb,) * 3, h, dt, cpml_cells=20, nt_max=nt, nrec_max=len(rec), device=dev)
        big.set_model(torch.from_numpy(vb).to(dev))
        big.set_cpml(R=1e-8, c_ref=cmax)
        big.inject(src + margin, torch.from_numpy(wav).to(dev))
        big.record(rec + margin)
        big.step(nt)
        big.sync()
        ref = big.traces.clone()
        big.close()
        del big
        torch.cuda.empty_cache()
        e_ref = misfit_flat(ref, torch.zeros_like(ref))
        out = {}
        for name, cells in (("learned_6", 6), ("polynomial_6", 6), ("polynomial_20", 20)):
            sim = Fdtd((n,) * 3, h, dt, cpml_cells=cells, nt_max=nt, nrec_max=len(rec), device=dev)
            sim.set_model(torch.from_numpy(vel).to(dev))
            if name == "learned_6":
                model.set_conditions(cmax, dt, f0)
                ska, _ = model.ska()
                sim.set_cpml_ska(ska)
            else:
                sim.set_cpml(R=1e-8, kappa_max=5.0, alpha_frac=0.05, q=3, c_ref=cmax)
            sim.inject(src, torch.from_numpy(wav).to(dev))
            sim.record(rec)
            secs = _timed(sim.stream, lambda: sim.step(nt))
            r = (sim.misfit(ref) / e_ref) ** 0.5
            out[name] = {"reflection": round(r, 5), "Mpoints_s": round(n ** 3 * nt / secs / 1e6, 1)}
            sim.close()
            del sim
            torch.cuda.empty_cache()
        out["learned_beats_polynomial_6"] = out["learned_6"]["reflection"] < out["polynomial_6"]["reflection"]
        evals[f"{f0:g}Hz"] = out
    train = {f"{f:.2f}Hz": {"polynomial_6": round(p, 5), "learned_6": round(l, 5)}
             for f, p, l in zip(res["f0"], res["poly_eval"], res["learned_eval"])}
    return {"workload": f"train 96^3 homogeneous c=2000 (8 shots per group, f0 groups {[round(f, 2) for f in res['f0']]} "
                        f"Hz from 5-30 Hz, incidence 0-80 deg, {iters} Adam steps); evaluate 512^3 layered seed 5, "
                        f"1000 steps at {list(eval_freqs)} Hz",
            "train_s": round(t_train, 1), "train_f0_range_hz": [5.0, 30.0], "train_angle_range_deg": [0.0, 80.0],
            "heldout_train_grid": train, "eval": evals,
            "learned_beats_polynomial_6_everywhere": all(v["learned_beats_polynomial_6"] for v in evals.values())}


# ----------------------------------------------------------------------------
# the FP64 oracle (CPU baseline and reference arm)
# ----------------------------------------------------------------------------
def oracle_sample(preset: str, nsteps: int, warm: int = 0):
    """Time the oracle on the full grid of the workload for nsteps time steps
    (after `warm` untimed ones).  Returns (Mpoints/s, seconds, threads)."""
    from oracle import oracle as O
    from paper_2606_06910_gb300 import synth
    w = synth.preset(preset)
    vel = w.velocity().astype(np.float64)
    g = O.Grid(vel * vel, w.h, w.dt, O.make_profiles(w.shape, w.cpml_cells, w.h, w.dt, w.c_max, R=w.R))
    st = O.State(w.shape)
    src = tuple(w.sources()[0])
    wav = synth.ricker(max(nsteps + warm, 1), w.dt, w.f0)
    if warm:
        O.run(g, st, warm, 0, src, wav)
    t = time.perf_counter()
    O.run(g, st, nsteps, warm, src, wav)
    dt = time.perf_counter() - t
    return float(np.prod(w.shape)) * nsteps / dt / 1e6, dt, int(O.threads())


def physical_cores() -> int:
    """Distinct (package, core) pairs of the host's CPUs (logical CPUs when
    the topology is not readable)."""
    import re
    base, seen = "/sys/devices/system/cpu", set()
    try:
        for d in os.listdir(base):
            if re.fullmatch(r"cpu\d+", d):
                try:
                    core = open(f"{base}/{d}/topology/core_id").read().strip()
                    pkg = open(f"{base}/{d}/topology/physical_package_id").read().strip()
                    seen.add((pkg, core))
                except OSError:
                    pass
    except OSError:
        pass
    return len(seen) or (os.cpu_count() or 1)


def oracle_sample_one_core(preset: str, nsteps: int = 1):
    """The oracle on one thread, in a child process (OpenMP fixes its thread
    count at load time): (Mpoints/s, seconds) or None."""
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", f"{preset}:{nsteps}"],
                           env=env, capture_output=True, text=True, timeout=600)
        d = json.loads(r.stdout.strip().splitlines()[-1])
        return d["mpts"], d["secs"]
    except Exception:
        return None


def oracle_accuracy_reference(store=None):
    """The FP64 oracle on the precision form's 128^3 accuracy instance: the
    pressure after each checkpoint and the traces (the same receivers as
    storage_accuracy_gpu).  store = "f16" / "bf16" rounds every stored field
    as that form stores it (FP64 arithmetic): the storage format's own error."""
    from oracle import oracle as O
    from paper_2606_06910_gb300 import synth
    w = synth.preset("layered128")
    vel = w.velocity().astype(np.float64)
    g = O.Grid(vel * vel, w.h, w.dt, O.make_profiles(w.shape, w.cpml_cells, w.h, w.dt, w.vmax, R=w.R),
               store=store, scale_p=1024.0 if store == "f16" else 1.0, scale_v=float(w.vmax) if store else 1.0)
    st = O.State(w.shape)
    src = tuple(w.sources()[0])
    wav = w.wavelet()[0].astype(np.float64)
    rec = synth.receiver_grid(w.shape, w.cpml_cells, 6, 6, w.cpml_cells[4])
    out, t, trs = {}, 0, []
    for c in ACCURACY_CHECKPOINTS:
        trs.append(O.run(g, st, c - t, t, src, wav, rec))
        t = c
        out[c] = st["p"].copy()
    out["traces"] = np.concatenate(trs)
    return out


def _rel_l2(run, ref):
    def rl(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))
    e = {f"p_step{c}": rl(run[c], ref[c]) for c in ACCURACY_CHECKPOINTS}
    e["traces"] = rl(run["traces"], ref["traces"])
    return e


def accuracy_line(gpu, ref, budget, rounded=None):
    """Relative L2 of the GPU's pressure at each checkpoint and of its traces
    against the oracle, with whether each meets the budget; with `rounded`
    (the oracle with the form's storage rounding) also the error that the
    storage format alone causes."""
    e = _rel_l2(gpu, ref)
    out = {"instance": "layered128 (seed 3), 500 steps, vs the FP64 oracle",
           "rel_l2": {k: float(f"{v:.4e}") for k, v in e.items()},
           "budget": budget, "budget_met": {k: v <= budget for k, v in e.items()},
           "budget_met_all": all(v <= budget for v in e.values())}
    if rounded is not None:
        out["storage_rounding_floor"] = {k: float(f"{v:.4e}") for k, v in _rel_l2(rounded, ref).items()}
    return out


def state_gb(shape, storage):
    """Device bytes of the stepped state: p and v in two sets plus the FP32 K table."""
    es = 4 if storage == "f32" else 2
    return (8 * es + 4) * float(np.prod(shape)) / 1e9


def workload_config(args, shape, cells, nt, world):
    cdesc = f"{cells[0]} cells" if len(set(cells)) == 1 else f"cells {','.join(map(str, cells))} (-x,+x,-y,+y,-z,+z)"
    out = {"workload": f"{args.preset}: {shape[0]}^3 layered 1500-4500 m/s, CPML {cdesc}, "
                       f"R=1e-8, 10 Hz Ricker, {nt} time steps per bench step",
           "grid": list(shape), "time_steps_per_step": nt, "cpml_cells": list(cells),
           "storage": args.storage, "parallelism": f"replicas x{world}",
           "l2": f"inputs larger than L2 (state {state_gb(shape, args.storage):.1f} GB per replica, L2 129 MB)"}
    if getattr(args, "variant", "plain") != "plain":
        out["variant"] = args.variant
    return out


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle on the host cores, on the same
    workload; each bench step is a bounded sample of it (one time step of the
    full grid)."""
    if rank != 0:
        return None
    import oracle
    from oracle import oracle as O
    from paper_2606_06910_gb300 import synth
    oracle.build()
    w = synth.preset(args.preset)
    cells = w.cpml_cells if args.cells is None else args.cells
    nt = args.nt or w.nt
    vel = w.velocity().astype(np.float64)
    g = O.Grid(vel * vel, w.h, w.dt, O.make_profiles(w.shape, cells, w.h, w.dt, w.c_max, R=w.R))
    st = O.State(w.shape)
    src = tuple(w.sources()[0])
    wav = synth.ricker(args.warmup + args.steps + 1, w.dt, w.f0)
    times = []
    for k in range(args.warmup + args.steps):
        t = time.perf_counter()
        O.run(g, st, 1, k, src, wav)
        if k >= args.warmup:
            times.append(time.perf_counter() - t)
    threads = int(O.threads())
    value = float(np.prod(w.shape)) * len(times) / sum(times) / 1e6
    sample = f"{args.preset} full grid, one FP64 oracle time step per bench step (OpenMP, {threads} threads)"
    return {
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * sum(times) / len(times), 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, w.shape, cells, nt, world),
        "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def cpu_baseline_leg(args, out, local):
    """The FP64 oracle on the host cores, after every GPU measurement: the
    timed sample of the workload (all threads, and one thread), and the
    oracle's run of the precision form's 128^3 accuracy instance, against
    which the FP32 path and the 16-bit forms report their relative L2 error."""
    import oracle
    from oracle import oracle as O
    oracle.build()
    nsamp = 8
    mpts, secs, threads = oracle_sample(args.preset, nsamp, warm=1)
    one = oracle_sample_one_core(args.preset, 1)
    line = {"value": round(mpts, 3), "unit": UNIT, "cores": int(O.threads()), "kind": "oracle",
            "sample": f"{args.preset} full grid, {nsamp} FP64 oracle time steps after 1 untimed ({secs:.1f} s)",
            "logical_cpus": os.cpu_count(), "physical_cores": physical_cores()}
    if one is not None:
        line["one_thread"] = {"value": round(one[0], 3), "unit": UNIT,
                              "sample": f"{args.preset} full grid, 1 FP64 oracle time step on one thread ({one[1]:.1f} s)"}
    forms = out.get("forms", {})
    if args.accuracy and "value" in out:
        import torch
        dev = torch.device("cuda", local)
        t0 = time.perf_counter()
        ref = oracle_accuracy_reference()
        line["accuracy_reference_s"] = round(time.perf_counter() - t0, 1)
        out["accuracy"] = accuracy_line(storage_accuracy_gpu(dev, "f32"), ref, 1e-4)
        for st in ("f16", "bf16"):
            if st in forms and "error" not in forms[st]:
                forms[st]["accuracy"] = accuracy_line(storage_accuracy_gpu(dev, st), ref, 2e-2,
                                                      oracle_accuracy_reference(st))
    return line


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.oracle_sample:
        preset, n = args.oracle_sample.split(":")
        mpts, secs, threads = oracle_sample(preset, int(n))
        print(json.dumps({"mpts": mpts, "secs": secs, "threads": threads}), flush=True)
        return
    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    out = {} if args.forms_only else run_ours(args, rank, world, local)
    if rank == 0 and world == 1 and args.forms:
        import torch
        dev = torch.device("cuda", local)
        forms = {}
        for f in [x for x in args.forms.split(",") if x]:
            torch.cuda.empty_cache()
            try:
                if f in ("f16", "bf16"):
                    forms[f] = form_storage(f, dev)
                elif f == "adjoint":
                    forms[f] = form_adjoint(dev)
                elif f.startswith("adjoint:"):
                    _, ns, nt = f.split(":")
                    forms[f] = form_adjoint(dev, nt=int(nt), nshots=int(ns), every=int(nt))
                elif f == "learned":
                    forms[f] = form_learned(dev)
                elif f == "cpml_overhead":
                    forms[f] = form_cpml_overhead(dev)
                elif f == "tblock":
                    forms[f] = form_tblock(dev)
                elif f == "decomp":
                    forms[f] = form_decomp(dev)
                elif f == "density":
                    forms[f] = form_density(dev)
                elif f == "staggered":
                    forms[f] = form_staggered(dev)
                elif f == "local_cpml":
                    forms[f] = form_local_cpml(dev)
                elif f == "aniso2d":
                    forms[f] = form_aniso2d(dev)
            except Exception as e:  # report, keep the main line
                forms[f] = {"error": f"{type(e).__name__}: {e}"[:300]}
        out["forms"] = forms
    if args.forms_only:
        if rank == 0:
            print(json.dumps(out), flush=True)
        return
    if rank == 0:
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline_leg(args, out, local)
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
