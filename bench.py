"""Benchmark of the MMC hot path on GB300: cell-updates per second.

One step = 100 MMC iterations (the cone-adaptation window, Sec. II) of the
whole batch: per iteration the FFT demag field (Eq. 14), the red and the black
sublattice pass; the window/adaptation kernel after the 100th.  The default
workload is the chiral-film temperature scan: 16 chains of 512x512x1 cells
(2x2x1 nm), DMI, perpendicular anisotropy, demag, T = 50 + 40 c K, random
initial state, all chains in one CUDA graph per step.

Printed (one JSON line): value = cell-updates/s with inputs resident in HBM
(device-timed with CUDA events on the library's stream); e2e = the same metric
through the public API with the state copied from pinned host memory and the
observables read back every step; roofline of the dominant kernel (per-kernel
CUDA-event durations from mmc_phase_times); cpu_baseline = the FP64 oracle on
the host cores on a bounded sample; clocks sampled with nvidia-smi during the
timed region.

--impl reference times the FP64 oracle itself (the reference arm of this
benchmark) on the same workload: each step is one iteration of one chain.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import re
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "MMC cell-updates/s incl. demag"
UNIT = "cell-updates/s"
SWEEPS_PER_STEP = 100
LOOP_SWEEPS = 5000          # iterations per field of the hysteresis-loop workload


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="chiral512",
                    choices=["chiral512", "chiral512_periodic", "film256", "film256_loop", "permalloy32",
                             "granular", "probe8192"])
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-demag", action="store_true", help="demag FFT convolution in FP64")
    ap.add_argument("--ff-demag", action="store_true",
                    help="demag FFT convolution in float-float (pairs of FP32 values on the FP32 pipe)")
    ap.add_argument("--fft-variant", type=int, default=0, choices=(0, 1, 2, 3, 4),
                    help="FP32 2D demag kernels: 0 timed pick at create, 1 radix 16, 2 radix 32, "
                         "3 radix 16 two blocks per SM, 4 warp 32x32 transforms (1024-point grids)")
    ap.add_argument("--stream-groups", type=int, default=0,
                    help="chain groups iterating on concurrent streams: 0 auto (2), 1 one stream")
    ap.add_argument("--sweep-tiles", type=int, default=0, choices=(0, 1),
                    help="1 banded pass on shared-memory halo tiles where the batch allows it, 0 per-block pass")
    ap.add_argument("--fuse-passes", type=int, default=1, choices=(0, 1),
                    help="1 black pass fused with the next forward row transforms where the batch allows it")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the cuFFT demag timing and the one-chain-per-launch comparison")
    ap.add_argument("--chains", type=int, default=0, help="use only the first N chains of the workload")
    ap.add_argument("--profile-run", type=int, default=0,
                    help="profiling case: run N iterations eagerly (no graphs, no timing) and exit")
    return ap.parse_args()


def workload(name):
    if name == "chiral512":
        return W.chiral512_batch(16, 512), True, "16 chains 512x512x1, 2x2x1 nm, DMI+Ku+demag, T=50..650 K"
    if name == "chiral512_periodic":
        return ([W.chiral_periodic(512, 50.0 + 40.0 * c, 10) for c in range(16)], True,
                "16 chains 512x512x1 periodic in-plane (exchange, DMI and demag, 10 images per side), "
                "2x2x1 nm, DMI+Ku, T=50..650 K")
    if name == "film256":
        return [W.film256(256)], True, "256x256x1, 4 nm, demag, B=100 mT"
    if name == "film256_loop":
        return ([W.film256(256)], True,
                "256x256x1, 4 nm, demag; hysteresis loop of 41 fields +100 -> -100 mT along x, "
                f"{LOOP_SWEEPS} iterations per field (one field per step), snapshot every 50 iterations")
    if name == "permalloy32":
        return [W.permalloy32()], False, "32x32x1 periodic, 5 nm, no demag"
    if name == "granular":
        sizes = W.granular_sizes(32, 7)
        return W.granular_batch(32, 7, sizes), True, "32 granular chains, sides %d..%d, hotspot, demag" % (
            min(sizes), max(sizes))
    if name == "probe8192":
        return [W.probe(8192)], False, "8192x8192x1, 5 nm, no demag"
    raise ValueError(name)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def nvtx_range(name):
    """Open (name) or close (None) an NVTX range, where torch provides NVTX."""
    import torch
    try:
        if name is None:
            torch.cuda.nvtx.range_pop()
        else:
            torch.cuda.nvtx.range_push(name)
    except (AttributeError, RuntimeError):
        pass


KERNEL_SOURCES = ("k_sweep.cu", "k_demag.cu", "k_demag_il.cuh", "demag_il.h", "demag_args.cuh", "fft.cuh",
                  "fft_il.cuh", "trial.cuh", "philox.cuh", "mmc_internal.h", "k_demag_w32.cu", "fft_w32.cuh",
                  "tma.cuh")


def strip_comments(src):
    """C/C++ source without its comments and trailing blanks (the kernel sources
    hold no string literal with comment markers)."""
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return "\n".join(ln.rstrip() for ln in src.splitlines() if ln.strip())


def kernel_source_hash(read=None):
    """Hash of the code (comments excluded) of the timed kernels' sources: a
    recorded ncu figure is used only when it was taken on the same code."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        if read is None:
            with open(os.path.join(ROOT, "paper_2106_05593_gb300", "csrc", f)) as fh:
                txt = fh.read()
        else:
            txt = read(f)
        h.update(strip_comments(txt).encode())
    return h.hexdigest()[:16]


def recorded_traffic(kernel, workload_name, src_hash):
    """DRAM bytes per launch from a committed ncu summary, if taken on this source."""
    p = os.path.join(ROOT, "profiles", "dram_traffic_per_launch.txt")
    if not os.path.exists(p):
        return None
    for ln in open(p):
        t = ln.split()
        if len(t) >= 4 and not ln.startswith("#") and t[0] == kernel and t[1] == workload_name and t[2] == src_hash:
            return float(t[3])
    return None


# algorithmic bytes per cell per launch: what each kernel must read and write
def spectrum_bytes_per_cell(specs):
    """Bytes per cell of the FP32 half spectrum (3 components, complex): 24 for rows
    zero padded to >= 2 nx, 12 for rows transformed circularly (periodic demag
    along x with a power-of-two extent >= 8: half as many kx)."""
    tot = cells = 0.0
    for sp in specs:
        nx = sp["mesh"][0]
        circ = (sp.get("demag_images", 0) > 0 and sp["pbc"][0] and nx >= 8 and (nx & (nx - 1)) == 0)
        n = float(np.prod(sp["mesh"]))
        tot += n * (12.0 if circ else 24.0)
        cells += n
    return tot / cells


def algorithmic_bytes(kind, demag, percell, spec=24.0):
    if kind == "sweep_pass":     # per pass: half the cells updated; 48 B/cell-update (+48 per-cell table)
        return 0.5 * (48.0 if demag else 32.0) + (0.5 * 48.0 if percell else 0.0)
    if kind == "demag_rows_fwd":  # m read 16 B, three half-spectrum rows written (spec B)
        return 16.0 + spec
    if kind == "demag_cols":      # spectrum read and written, 2 x spec B
        return 2.0 * spec
    if kind == "demag_rows_inv":  # spectrum read (spec B), h_eff written 16 B
        return spec + 16.0
    if kind == "black_pass_rows_fwd":   # m read 16 B (both colours), black m written 8 B and black h_eff
        return 16.0 + 8.0 + 8.0 + spec  # read 8 B per cell (16 B per black cell), spectrum written
    if kind == "rows_inv_red_pass":     # spectrum read, m read 16 B (red cells and black neighbours),
        return spec + 16.0 + 8.0 + 8.0  # red m written 8 B and black h_eff written 8 B per cell
    return 0.0


CPU_SAMPLE_SIDE = 512      # the oracle's sample: at most 512 x 512 cells in-plane of chain 0
CPU_SAMPLE_IMAGES = 1      # periodic demag images of the oracle's sample


def crop_spec(spec, side=CPU_SAMPLE_SIDE):
    """The corner block of at most side x side cells (all layers) of a chain,
    per-cell arrays cut to match, so that the oracle's sample of a large chain
    stays bounded; the per-cell work of an iteration does not depend on the
    mesh size (the demag FFT's only by its log factor).  A periodic demag kernel
    is built with CPU_SAMPLE_IMAGES images per side: the oracle's kernel build
    grows with the images, its iterations do not (the same FFT convolution)."""
    nx, ny, nz = spec["mesh"]
    cx, cy = min(nx, side), min(ny, side)
    note = ""
    if spec.get("demag_images", 0) > CPU_SAMPLE_IMAGES:
        spec = dict(spec)
        spec["demag_images"] = CPU_SAMPLE_IMAGES
        note = f"{CPU_SAMPLE_IMAGES} periodic demag image(s) per side for the oracle's kernel build, "
    if (cx, cy) == (nx, ny):
        return spec, note + "chain 0"
    n = nx * ny * nz
    out = dict(spec)
    out["mesh"] = (cx, cy, nz)
    for k, v in spec.items():
        if isinstance(v, np.ndarray) and v.shape[:1] == (n,):
            out[k] = np.ascontiguousarray(v.reshape((nz, ny, nx) + v.shape[1:])[:, :cy, :cx].reshape((-1,) + v.shape[1:]))
    return out, note + "corner block of chain 0"


def host_description():
    """Host cores (nproc) and CPU model name (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model and os.path.exists("/proc/cpuinfo"):
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part")):
                model = ln.split(":", 1)[1].strip()
                break
    return {"host_cores": os.cpu_count(), "cpu_model": model}


def cpu_baseline(specs, demag, nsweeps=3):
    """FP64 oracle, one thread, one chain of the workload (its corner block
    when larger than 512 x 512 in-plane) for a few iterations."""
    import oracle as O
    spec, what = crop_spec(specs[0])
    o = O.Oracle(spec)
    n = o.n
    m = o.init_state(random=True, length=0.5, chain=0, seed=1)
    st = O.new_state(seed=1, theta_deg=30.0, adapt=True, demag_mode=1 if demag else 0)
    o.run(m, 1, st)
    t0 = time.perf_counter()
    o.run(m, nsweeps, st)
    dt = time.perf_counter() - t0
    return {"value": n * nsweeps / dt, "unit": UNIT, "cores": 1, "kind": "oracle", **host_description(),
            "sample": f"{what} of the workload "
                      f"({spec['mesh'][0]}x{spec['mesh'][1]}x{spec['mesh'][2]}), "
                      f"{nsweeps} iterations after 1 warm-up, demag {'FFT FP64' if demag else 'off'}"}


def replica_seed(rank):
    """Seed of rank's replica: every rank runs the whole workload as an
    independent replica (weak scaling), so the ranks draw different numbers."""
    return 1 + rank


def reduce_max(x, device):
    """Max of x over all ranks (identity without a process group); the device
    follows the backend (CUDA tensors for NCCL, CPU tensors for gloo)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(local_ms, units_per_rank, world, device):
    """Whole-job throughput: the units every rank processed over the slowest
    rank's time.  Returns (max ms, units / s)."""
    ms_max = reduce_max(local_ms, device)
    return ms_max, units_per_rank * world / (ms_max * 1e-3)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    specs, demag, desc = workload(args.workload)
    spec, what = crop_spec(specs[0])
    o = O.Oracle(spec)
    m = o.init_state(random=True, length=0.5, chain=0, seed=1)
    st = O.new_state(seed=1, theta_deg=30.0, adapt=True, demag_mode=1 if demag else 0)
    per = 1
    for _ in range(args.warmup):
        m, _, _ = o.run(m, per, st)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        m, _, _ = o.run(m, per, st)
    dt = time.perf_counter() - t0
    value = o.n * per * args.steps / dt
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "description": desc,
                       "sample": f"{what} "
                                 f"({spec['mesh'][0]}x{spec['mesh'][1]}x{spec['mesh'][2]}), "
                                 "one MMC iteration per step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", **host_description(),
                             "sample": f"{what} of {args.workload} "
                                       f"({spec['mesh'][0]}x{spec['mesh'][1]}x{spec['mesh'][2]}), "
                                       f"{per} iteration per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def demag_prec(args):
    """mmc_options.demag_fp64 of the run: 0 FP32, 1 FP64, 2 float-float."""
    return 2 if args.ff_demag else int(args.fp64_demag)


def fp64_demag_compare(MMC, specs, seed, stream, cells_per_step, steps=2, prec=1):
    """The workload with its demag FFT convolution accumulated at FP64 precision
    (prec 1: FP64; prec 2: float-float on the FP32 pipe), the sweep in FP32:
    whole-batch rate over `steps` steps, the demag update time, and the largest
    difference of the Eq. 5 decision values (kT) of one pass of chain 0 between
    the FP32 and this convolution on the same state (the FP64 and float-float
    fields equal the oracle's to 1e-9 and 1e-10 of max |H| in the parity tests)."""
    import torch
    g64 = MMC(specs, demag=1, demag_fp64=prec, stream=stream)
    g64.init_random(seed)
    g64.sweep(SWEEPS_PER_STEP, seed)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        g64.sweep(SWEEPS_PER_STEP, seed)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    ph = g64.phase_times(10, seed)
    upd = sum(ph[k][0] for k in ("demag_rows_fwd", "demag_cols", "demag_rows_inv")) / max(ph["demag_cols"][1], 1)
    m4 = g64.get_m(0)
    g32 = MMC(specs[:1], demag=1, stream=stream)
    g1 = MMC(specs[:1], demag=1, demag_fp64=prec, stream=stream)
    dd = 0.0
    for color in (0, 1):
        decs = []
        for gg in (g32, g1):
            gg.set_m(m4)
            decs.append(gg.pass_debug(0, color, 7, seed, 20.0)[0])
        dd = max(dd, float(np.abs(decs[0].astype(np.float64) - decs[1]).max()))
    return {"value": cells_per_step * steps / (ms * 1e-3), "unit": UNIT, "steps": steps,
            "demag_update_ms": upd,
            "decision_value_max_diff_fp32_vs_%s_kT" % ("fp64" if prec == 1 else "float_float"): dd}


def batched_plain_identity(MMC, specs, demag, args, variant, seed, stream, iters=100):
    """Batched and plain forms at equal accuracy: one-chain contexts given
    chain_base = k run chain k's Markov chain; after `iters` iterations from the
    same random start every chain's state equals the batch's bit for bit."""
    b = MMC(specs, demag=int(demag), demag_fp64=demag_prec(args), fft_variant=variant, stream=stream)
    b.init_random(seed)
    b.sweep(iters, seed)
    same = 0
    for k, sp in enumerate(specs):
        p = MMC([sp], demag=int(demag), demag_fp64=demag_prec(args), fft_variant=variant, chain_base=k,
                stream=stream)
        p.init_random(seed)
        p.sweep(iters, seed)
        same += int(np.array_equal(p.get_m(0), b.get_m(k)))
        p.close()
    return {"identical_chains": same, "chains": len(specs), "iterations": iters,
            "note": "plain context k with chain_base = k is chain k of the batch (same random numbers)"}


def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2106_05593_gb300 import MMC, build
    build.build()
    specs, demag, desc = workload(args.workload)
    if args.chains > 0:
        specs = specs[:args.chains]
        desc += f" (first {len(specs)} chains)"
    percell = args.workload == "granular"
    stream = torch.cuda.Stream()
    if args.profile_run > 0:
        gp = MMC(specs, demag=int(demag), demag_fp64=demag_prec(args), use_graphs=0,
                 fft_variant=args.fft_variant, sweep_tiles=args.sweep_tiles, stream_groups=args.stream_groups,
                 fuse_passes=args.fuse_passes, stream=stream)
        gp.init_random(replica_seed(rank))
        gp.sweep(args.profile_run, replica_seed(rank))
        torch.cuda.synchronize()
        print("profile run ok", gp.launches, flush=True)
        return
    g = MMC(specs, demag=int(demag), demag_fp64=demag_prec(args), fft_variant=args.fft_variant,
            stream_groups=args.stream_groups, sweep_tiles=args.sweep_tiles, fuse_passes=args.fuse_passes,
            stream=stream)
    seed = replica_seed(rank)
    g.init_random(seed)
    ncell = sum(g.ncell)
    loop = args.workload == "film256_loop"
    sweeps_per_step = LOOP_SWEEPS if loop else SWEEPS_PER_STEP
    cells_per_step = ncell * sweeps_per_step
    fields = W.hysteresis_fields(41)
    step_no = [0]

    def do_step():
        """One step: 100 iterations of the batch, or for the loop workload the
        next field of the loop and its iterations with snapshots."""
        if loop:
            g.set_field(fields[step_no[0] % len(fields)])
            g.sweep_sampled(LOOP_SWEEPS, seed, 50)
        else:
            g.sweep(SWEEPS_PER_STEP, seed)
        step_no[0] += 1

    for _ in range(args.warmup):
        do_step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.4)
    barrier()
    torch.cuda.synchronize()
    l0 = g.launches
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    nvtx_range("timed_steps")            # lets a profiler select the timed launches
    e0.record(stream)
    for _ in range(args.steps):
        do_step()
    e1.record(stream)
    torch.cuda.synchronize()
    nvtx_range(None)
    barrier()
    ms = e0.elapsed_time(e1)
    launches = g.launches - l0
    clk = clocks.stop()
    ms_max, value = job_throughput(ms, cells_per_step * args.steps, world, "cuda")

    # per-kernel durations (CUDA events on the library's stream), one more window
    phases = g.phase_times(SWEEPS_PER_STEP, seed)
    peak, peak_kind = measured_peaks()
    best = None
    for kind, (tms, cnt) in phases.items():
        if cnt and (best is None or tms > phases[best][0]):
            best = kind
    tms, cnt = phases[best]
    avg_s = tms / cnt * 1e-3
    # FP64 and float-float spectra hold 16 B per complex value, FP32 8 B
    spec_b = spectrum_bytes_per_cell(specs) * (2.0 if demag_prec(args) else 1.0)
    bytes_per_launch = algorithmic_bytes(best, demag, percell, spec_b) * ncell
    achieved = bytes_per_launch / avg_s / 1e9
    src = kernel_source_hash()
    roofline = {"bound": "hbm", "kernel": best, "achieved": achieved, "peak": peak,
                "peak_kind": f"{peak_kind} copy bandwidth", "unit": "GB/s", "frac": achieved / peak,
                "traffic": recorded_traffic(best, args.workload, src),
                "algorithmic_bytes_per_launch": bytes_per_launch, "avg_launch_ms": avg_s * 1e3}
    # the sublattice pass and the three demag kernels on their own: with the fused
    # path they run inside the fused kernels, so a context without the fusion times them
    fused = phases["black_pass_rows_fwd"][1] > 0
    ph_unfused = phases
    if fused:
        gu = MMC(specs, demag=int(demag), fuse_passes=0, fft_variant=g.fft_tuning()[0], stream=stream)
        gu.init_random(seed)
        gu.sweep(SWEEPS_PER_STEP, seed)
        ph_unfused = gu.phase_times(SWEEPS_PER_STEP, seed)
        del gu
    sweep_ms, sweep_cnt = ph_unfused["sweep_pass"]
    sweep_bytes = algorithmic_bytes("sweep_pass", demag, percell) * ncell
    sweep_roof = {"kernel": "sublattice pass" + (" (unfused context)" if fused else ""),
                  "achieved": sweep_bytes / (sweep_ms / sweep_cnt * 1e-3) / 1e9, "peak": peak,
                  "frac": sweep_bytes / (sweep_ms / sweep_cnt * 1e-3) / 1e9 / peak, "unit": "GB/s",
                  "avg_launch_ms": sweep_ms / sweep_cnt}

    # comparisons: demag update through cuFFT, and the same chains one per context
    compare = None
    if not args.no_compare:
        compare = {}
        if demag:
            kinds = ("demag_rows_fwd", "demag_cols", "demag_rows_inv")
            own = sum(ph_unfused[k][0] for k in kinds) / max(ph_unfused["demag_cols"][1], 1)
            cf = MMC(specs, demag=1, demag_cufft=1, demag_fp64=demag_prec(args), stream=stream)
            cf.init_random(seed)
            ph = cf.phase_times(20, seed)
            # one demag update per iteration; the cuFFT path records one mark per
            # padded-size group, so divide by the updates, not by the marks
            cfm = sum(ph[k][0] for k in kinds) / 20.0
            compare["demag_update_ms"] = {"own": own, "cufft": cfm}
            if not demag_prec(args):
                compare["fp64_demag"] = fp64_demag_compare(MMC, specs, seed, stream, cells_per_step)
                compare["demag_update_ms"]["own_fp64"] = compare["fp64_demag"]["demag_update_ms"]
                compare["ff_demag"] = fp64_demag_compare(MMC, specs, seed, stream, cells_per_step, prec=2)
                compare["demag_update_ms"]["own_float_float"] = compare["ff_demag"]["demag_update_ms"]
            v, tms = g.fft_tuning()
            tu = g.tuning()
            compare["autotune"] = {"stream_groups": tu["stream_groups"], "from_cache": tu["from_cache"],
                                   "iteration_ms_by_groups": {"1": tu["groups_ms"][0], "2": tu["groups_ms"][1],
                                                              "3": tu["groups_ms"][2]}}
            compare["fft_variant"] = {"picked": {0: None, 1: "radix16", 2: "radix32", 3: "radix16x2", 4: "warp32x32"}[v],
                                      "create_time_ms": {"radix16": tms[0], "radix32": tms[1],
                                                         "radix16x2": tms[2], "warp32x32": tms[3]}}
            del cf
        if len(specs) > 1:
            # the plain form runs the kernels the batch runs (its FFT variant), so that
            # the two forms differ only in how the chains are launched
            plain = [MMC([sp], demag=int(demag), demag_fp64=demag_prec(args), fft_variant=g.fft_tuning()[0],
                         stream=stream) for sp in specs]
            for k, p1 in enumerate(plain):
                p1.set_m(g.get_m(k))
                p1.sweep(SWEEPS_PER_STEP, seed)
            torch.cuda.synchronize()
            steps_p = max(1, min(args.steps, 3))
            p0 = torch.cuda.Event(enable_timing=True)
            p1e = torch.cuda.Event(enable_timing=True)
            p0.record(stream)
            for _ in range(steps_p):
                for p1 in plain:
                    p1.sweep(SWEEPS_PER_STEP, seed)
            p1e.record(stream)
            torch.cuda.synchronize()
            pms = p0.elapsed_time(p1e)
            compare["plain_one_chain_per_launch"] = {
                "value": cells_per_step * steps_p / (pms * 1e-3), "unit": UNIT, "steps": steps_p,
                "batched_over_plain": value / world / (cells_per_step * steps_p / (pms * 1e-3)),
                "agreement": batched_plain_identity(MMC, specs, demag, args, g.fft_tuning()[0], seed, stream)}
            del plain

    # end to end through the public API: state from pinned host memory, observables back
    e2e = None
    if args.e2e_steps > 0:
        # every chain's state in one pinned host buffer, set with one call; every
        # chain's observables read back with one call
        buf = torch.empty((int(sum(g.ncell)), 4), dtype=torch.float32, pin_memory=True)
        buf.copy_(torch.from_numpy(g.get_m_all()))
        host_m = buf.numpy()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        d2h = 0
        for _ in range(args.e2e_steps):
            g.set_m_all(host_m)
            do_step()
            for ob in g.observables_all():
                d2h += 8 * (3 + 2) + 8 * ob["hist"].size
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        _, e2e_value = job_throughput(1e3 * dt, cells_per_step * args.e2e_steps, world, "cuda")
        e2e = {"value": e2e_value, "unit": UNIT,
               "h2d_bytes_per_step": int(host_m.nbytes),
               "d2h_bytes_per_step": int(d2h // args.e2e_steps)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(specs, demag)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {0: "f32", 1: "f32 (demag FFT f64)", 2: "f32 (demag FFT float-float)"}[demag_prec(args)],
            "data": "synthetic",
            "config": {"workload": args.workload, "description": desc, "cells": ncell,
                       "sweeps_per_step": sweeps_per_step, "demag": "once per iteration" if demag else "off",
                       "l2": "working set larger than L2" if args.workload in ("chiral512", "chiral512_periodic", "granular", "probe8192")
                       else "working set L2-resident (no flush)", "graphs": True},
            "roofline": roofline, "roofline_sweep_pass": sweep_roof, "compare": compare,
            "phases_ms": {k: round(v[0] / max(v[1], 1), 5) for k, v in phases.items()},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
            "kernel_source": src,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
