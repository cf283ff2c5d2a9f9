#!/usr/bin/env python3
"""Throughput of the PSR-NQS hot path on GB300: log psi forward + reverse-scan
backward (per-sample O_k) + local energy over every bond-flip-connected
configuration, 2D Heisenberg 52x52 OBC, hidden 128, 3 layers, 4096 samples,
BF16 projections with FP32 scan.

One step = psr_logpsi(samples) + psr_grad(samples, O_k per sample)
         + psr_local_energy(samples) through the C ABI.
Unit = one (configuration, site) pair of a forward pass, counting the samples
and every connected configuration with all N sites ("logical"); the sites the
library actually evaluates (connected forwards resume at the chunk holding
the first flipped site) are reported beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank runs its own 4096 samples on its own GPU (weak
scaling, no data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "configs·sites/s for log psi fwd+bwd+E_loc at 52x52, BF16 vs FP32; % HBM roofline"
UNIT = "configs·sites/s"
N_LAYERS, HIDDEN = 3, 128
MMA_FLOPS_PER_SITE = 2 * HIDDEN * HIDDEN * 9  # nine HxH products per site (BF16 path)
CHUNK_BF16 = 32

WORKLOADS = {
    # name: (Lx, Ly, samples)
    "heisenberg_52x52": (52, 52, 4096),
    "heisenberg_52x52_small": (52, 52, 64),     # profiling-sized case of the same kernel
    "heisenberg_10x10": (10, 10, 16384),
}

# kernels launched per call of each entry point (BF16 precision)
LAUNCHES = {"logpsi": 4, "local_energy": 11}
TC_STASH_BUDGET = 16 << 30      # bytes of stash and layer arrays per gradient batch


def grad_launches(n, L, nL=N_LAYERS, H=HIDDEN):
    """Kernels of one tensor-core gradient call: three packing kernels, then per
    batch 3 nL forward launches (scan and output map per layer, projections
    above layer 0, the readout adjoint) and 4 nL - 1 backward launches."""
    npad = (L + 63) & ~63
    per = ((nL * 4 * H + 1) * npad + 7 * H * npad) * 4
    B = max(1, min(n, TC_STASH_BUDGET // per))
    return 3 + -(-n // B) * (7 * nL - 1)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--workload", default="heisenberg_52x52", choices=sorted(WORKLOADS))
    ap.add_argument("--fp32-samples", type=int, default=64)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--no-scan", action="store_true")
    ap.add_argument("--no-sample", action="store_true")
    ap.add_argument("--no-2d", action="store_true")
    ap.add_argument("--no-lru", action="store_true")
    ap.add_argument("--no-vmc", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--depth-only", action="store_true",
                    help="only the fused-forward latency versus sample count, beside the parallel scan")
    ap.add_argument("--sample-only", action="store_true",
                    help="only the sampler leg (profiling runs)")
    ap.add_argument("--sample-n", type=int, default=0,
                    help="samples of the sample-only run (default: the workload's samples)")
    ap.add_argument("--mixed-only", action="store_true",
                    help="only the mixed-lattice batch leg")
    ap.add_argument("--samples-2d", type=int, default=64,
                    help="samples of the 2D patched-model leg (52x52; FP16 tensor cores, FP32 on 8 of them)")
    ap.add_argument("--scan-only", action="store_true",
                    help="only the standalone scan measurement (profiling runs)")
    ap.add_argument("--scan-n", type=int, default=0,
                    help="sequences of the scan-only run (default: the workload's samples)")
    ap.add_argument("--scan-tile", default="",
                    help="units,chunk: fixed tile shape of the scan-only run (default: autotuned)")
    ap.add_argument("--model2d-only", action="store_true",
                    help="only the 2D patched-model leg (52x52, --samples-2d samples)")
    ap.add_argument("--lru-only", action="store_true",
                    help="only the deep 1D LRU leg (TFIM chain N = 256, --samples-lru samples)")
    ap.add_argument("--samples-lru", type=int, default=1024,
                    help="samples of the deep 1D LRU leg")
    ap.add_argument("--paper2d-only", action="store_true",
                    help="only the 2D VMC step at the paper's 2D configuration")
    ap.add_argument("--paper2d-sizes", default="10,20",
                    help="lattice sides L of the paper-configuration 2D leg")
    ap.add_argument("--paper2d-reps", type=int, default=2)
    ap.add_argument("--paper2d-warmup", type=int, default=1,
                    help="untimed steps before the timed ones (the sampler is tuned in any case)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--fwd-shape", type=int, default=0,
                    help="BF16 forward shape: sequences per MMA stream (1 or 2); 0 = the library's choice")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_samples(rank, n, Lx, Ly):
    """The samples of one rank: every rank draws its own n configurations
    (seed 1000 + rank), so per-GPU work is fixed as ranks are added."""
    from paper_2605_13807_gb300 import inputs
    return inputs.neel_like_spins(1000 + rank, n, Lx, Ly)


def reduce_over_ranks(x, op, world, device):
    """all_reduce of one float over the ranks (op "max" or "sum"); the value
    itself when running alone."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_rate(units_this_rank, ms_this_rank, world, device):
    """Whole-job throughput: the units all ranks processed divided by the
    slowest rank's time (max over ranks).  Returns (units/s, max ms)."""
    units = reduce_over_ranks(units_this_rank, "sum", world, device)
    ms = reduce_over_ranks(ms_this_rank, "max", world, device)
    return units / (ms / 1e3), ms


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"psr_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = max((num(r[2]) for r in rows if num(r[2]) is not None), default=None)
        power = [num(r[3]) for r in rows if num(r[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        loaded = [s for s, p in zip(sm, power) if p is not None and p > 0.3 * max(power)] or sm
        loaded.sort()
        return {"sm_mhz": loaded[len(loaded) // 2] if loaded else None, "sm_max_mhz": smax,
                "reasons": reasons, "samples": len(rows)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def kernel_hash(src_name="psr_fwd_bf16.cu"):
    src = os.path.join(ROOT, "paper_2605_13807_gb300", "csrc", src_name)
    return hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]


def profiled_traffic_per_unit(profile="fwd_bf16_connected_52x52.md", src_name="psr_fwd_bf16.cu",
                              key="dram bytes per evaluated config-site"):
    """DRAM bytes per unit of work of a kernel, from its committed ncu
    summary, if the summary was taken of the current kernel source."""
    path = os.path.join(ROOT, "profiles", profile)
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if line.startswith("- ") and ":" in line:
            k, v = line[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel source sha256/16") != kernel_hash(src_name):
        return None
    try:
        return float(vals[key])
    except (KeyError, ValueError):
        return None


# ------------------------------------------------------------- reference arm

def oracle_rate(Lx, Ly, seconds, threads=None):
    """The FP64 oracle (sequential recurrence) timed on the host cores over
    the step's three stages for one sample: its log psi and O_k (the
    oracle's reverse mode), and E_loc over k of its connected
    configurations (each a full sequential forward), k chosen so the run
    takes about `seconds`.  Units as in the GPU metric: (1 + k) logical
    configuration x site pairs.  Returns (config-sites/s, cores, sample
    description)."""
    import numpy as np

    from oracle import oracle as orc
    from paper_2605_13807_gb300 import inputs

    cores = threads or (os.cpu_count() or 1)
    N = Lx * Ly
    theta = inputs.glorot_params(N_LAYERS, HIDDEN, seed=0)
    s = inputs.neel_like_spins(1000, 1, Lx, Ly)
    offs, ent, diag = orc.connected(orc.HEISENBERG, Lx, Ly, False, s)
    sp = np.repeat(s, len(ent), axis=0)
    r = np.arange(len(ent))
    sp[r, ent[:, 1]] ^= 1
    sp[r, ent[:, 2]] ^= 1
    t0 = time.perf_counter()
    orc.logpsi(theta, N_LAYERS, HIDDEN, sp[:1], u1=True, threads=1)
    t1 = time.perf_counter() - t0
    t0 = time.perf_counter()
    lp_s, _ok = orc.grad(theta, N_LAYERS, HIDDEN, s, u1=True, threads=1)
    t_grad = time.perf_counter() - t0
    per_core = max(1, int(round(max(seconds - t_grad, t1) / max(t1, 1e-6))))
    k = min(len(sp), per_core * cores)
    t0 = time.perf_counter()
    lp_s, _ok = orc.grad(theta, N_LAYERS, HIDDEN, s, u1=True, threads=1)
    lp_c = orc.logpsi(theta, N_LAYERS, HIDDEN, sp[:k], u1=True, threads=cores)
    orc.eloc_combine(diag[0], orc.offdiag_coeff(orc.HEISENBERG), lp_s[0], lp_c)
    dt = time.perf_counter() - t0
    desc = (f"FP64 oracle on one {Lx}x{Ly} sample: log psi and O_k (reverse mode, 1 thread), then E_loc "
            f"over {k} of its {len(ent)} connected configurations (full sequential forwards, {cores} "
            f"threads); units (1 + {k}) x {N} sites in {dt:.1f} s")
    return (1 + k) * N / dt, cores, desc


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    Lx, Ly, n = WORKLOADS[args.workload]
    per_step = max(1.0, args.cpu_seconds / 3)
    for _ in range(args.warmup):
        oracle_rate(Lx, Ly, per_step / 4)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v, cores, desc = oracle_rate(Lx, Ly, per_step)
        vals.append(v)
    wall = time.perf_counter() - t0
    value = sum(vals) / len(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"heisenberg_{Lx}x{Ly}_obc_{n}_samples", "lattice": f"{Lx}x{Ly} OBC",
                   "samples_per_gpu": n, "hidden": HIDDEN, "layers": N_LAYERS,
                   "parallelism": "host threads (FP64 oracle on a bounded sample)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm

def scan_leg(args, n, N, dev, reps=5):
    """The standalone chunked scan (psr_scan) over one layer's worth of the
    workload: n sequences x N sites x 128 units, FP32 a, b -> h (12 bytes per
    element from HBM; 17 GB per launch at 52x52, far above L2).  The tile
    shape is picked by the context's autotuner on the first call."""
    import torch

    from paper_2605_13807_gb300 import api, binding as B, inputs
    ctx = B.context()
    B.psr_context_set_profiling(ctx, True)
    a, b, h0 = inputs.scan_inputs_device(7, n, N, HIDDEN, dev)
    h = torch.empty_like(a)
    forced = tuple(int(x) for x in args.scan_tile.split(",")) if args.scan_tile else None
    if forced is None:
        B.psr_context_set_autotune(ctx, True)
        api.scan(a, b, h0, out=h)
        B.psr_context_set_autotune(ctx, False)
        tile, tuned = B.psr_scan_tile_for(ctx, n, N, HIDDEN)
    else:
        tile, tuned = forced, False
    for _ in range(3):
        api.scan(a, b, h0, tile=forced, out=h)
    ms = []
    for _ in range(reps):
        api.scan(a, b, h0, tile=forced, out=h)
        ms.append(B.psr_context_stage_ms(ctx)["scan"])
    api.sync()
    elems = n * N * HIDDEN
    algo = 12 * elems + 4 * n * HIDDEN
    avg = sum(ms) / len(ms)
    peaks, src = measured_peaks()
    peak = float(peaks.get("hbm_gbs"))
    achieved = algo / (avg / 1e3) / 1e9
    tpe = profiled_traffic_per_unit("scan_52x52_layer.md", "psr_scan.cu",
                                    "dram bytes per element")
    del a, b, h0, h
    torch.cuda.empty_cache()
    return {"kernel": "scan_kernel (psr_scan, standalone chunked scan)",
            "shape": [n, N, HIDDEN], "tile": {"units": tile[0], "chunk": tile[1]},
            "tuned": tuned, "ms": avg,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": f"hbm_gbs of {src}",
                         "traffic": (tpe * elems if tpe is not None else None),
                         "algorithmic_bytes_per_launch": algo, "bytes_per_unit": 12}}


# FP32 CUDA-core peak derived from unit counts and clock: 152 SMs x 128 FP32
# lanes x 2 flops per FMA x 2.07 GHz (maximum SM clock).
FP32_SIMT_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def sample_leg(theta, n, N, dev, reps=2):
    """The exact autoregressive sampler (psr_sample) drawing n samples of N
    sites from the caller's uniforms; samples per CTA picked by the
    autotuner on the first call.  FP32 on CUDA cores: 18 H^2 flops per
    sample-site (the forward's products), against the derived FP32 peak."""
    import torch

    from paper_2605_13807_gb300 import api, binding as B, inputs
    ctx = B.context()
    B.psr_context_set_profiling(ctx, True)
    g = torch.Generator(device=dev)
    g.manual_seed(3)
    u = torch.rand((n, N), generator=g, device=dev, dtype=torch.float32)
    cfg = api.ModelConfig(N_LAYERS, HIDDEN, True, "fp32")
    api.set_autotune(True)
    s, lp = api.sample(theta, u, cfg)
    api.set_autotune(False)
    per_cta, tuned = B.psr_sample_tile_for(ctx, n, N, N_LAYERS, HIDDEN)
    ms = []
    for _ in range(reps):
        api.sample(theta, u, cfg, spins=s, logpsi=lp)
        ms.append(B.psr_context_stage_ms(ctx)["sample"])
    api.sync()
    avg = sum(ms) / len(ms)
    flops = n * N * MMA_FLOPS_PER_SITE
    achieved = flops / (avg / 1e3) / 1e12
    # the same draws' model at BF16: the tensor-core sampler (blocks of 32
    # samples as MMA columns; the chain of a site's MMA stages bounds it)
    cfg16 = api.ModelConfig(N_LAYERS, HIDDEN, True, "bf16")
    api.sample(theta, u, cfg16, spins=s, logpsi=lp)
    ms16 = []
    for _ in range(reps):
        api.sample(theta, u, cfg16, spins=s, logpsi=lp)
        ms16.append(B.psr_context_stage_ms(ctx)["sample"])
    api.sync()
    avg16 = sum(ms16) / len(ms16)
    del u, s, lp
    return {"kernel": "sample_kernel (psr_sample, exact autoregressive sampler, FP32)",
            "samples": n, "sites": N, "samples_per_cta": per_cta, "tuned": tuned, "ms": avg,
            "value": n * N / (avg / 1e3), "unit": "sample-sites/s",
            "roofline": {"bound": "alu", "achieved": achieved, "peak": FP32_SIMT_TFLOPS,
                         "unit": "TFLOP/s", "frac": achieved / FP32_SIMT_TFLOPS,
                         "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz",
                         "traffic": None, "flops_per_unit": MMA_FLOPS_PER_SITE},
            "bf16_tensor_cores": {"kernel": "sample_tc_kernel (BF16 operands, FP32 gates, scan, readout)",
                                  "ms": avg16, "value": n * N / (avg16 / 1e3), "unit": "sample-sites/s",
                                  "speedup_vs_fp32": avg / avg16}}


# FLOPs per evaluated patch of the 2D patched minGRU (3 layers, hidden H):
# layer 0: W_h h_V and C h (2 x 2H^2); layers 1, 2: W_z x, W_h x, W_h h_V,
# C h, D x (5 x 2H^2 each).
def flops_per_patch_2d(H):
    return 2 * H * H * 12


def model2d_leg(Lx, Ly, n, dev, reps=2, H=256, n32=8):
    """The paper's 2D patched minGRU at its 52x52 configuration (3 layers,
    d_h = 256, 2x2 patches): log psi of n samples plus E_loc over all their
    connected configurations, in the headline metric's unit (configuration x
    spin site, logical), on the tensor cores (FP16 operands, FP32
    accumulation, gates, scan and softmax); the FP32 CUDA-core path of the
    same model on n32 of the samples for comparison."""
    import torch

    from paper_2605_13807_gb300 import api, binding as B, inputs
    ham = B.make_hamiltonian("heisenberg", Lx, Ly, False, True, 1.0, 0.0)
    theta = torch.from_numpy(inputs.glorot_params2d(N_LAYERS, H, seed=0)).to(dev)
    N, Px, Py = Lx * Ly, Lx // 2, Ly // 2
    ctx = B.context()

    def run(prec, m):
        cfg = api.ModelConfig(N_LAYERS, H, True, prec)
        spins = torch.from_numpy(rank_samples(0, m, Lx, Ly)).to(dev)
        _, ent, _ = api.connected(spins, ham)
        E = int(ent.shape[0])
        r0 = (ent[:, 1].to(torch.int64) // Lx) // 2
        evaluated = m * Px * Py + int(((Py - r0) * Px).sum().item())
        lp = torch.empty(m, dtype=torch.float32, device=dev)
        el = torch.empty(m, dtype=torch.float32, device=dev)
        st = torch.empty(3, dtype=torch.float64, device=dev)

        def step():
            api.logpsi2d(theta, spins, cfg, Lx, Ly, out=lp)
            api.local_energy2d(theta, spins, cfg, ham, out=el, stats=st)

        step()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            step()
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / reps
        B.psr_context_set_profiling(ctx, True)
        api.local_energy2d(theta, spins, cfg, ham, out=el, stats=st)
        conn_ms = B.psr_context_stage_ms(ctx)["fwd_connected"]
        B.psr_context_set_profiling(ctx, False)
        conn_patches = evaluated - m * Px * Py
        achieved = conn_patches * flops_per_patch_2d(H) / (conn_ms / 1e3) / 1e12
        return {"samples": m, "connected": E, "value": (m + E) * N / (ms / 1e3), "unit": UNIT,
                "ms_per_step": ms, "evaluated_patches_per_step": evaluated, "connected_launch_ms": conn_ms,
                "achieved_tflops": achieved, "energy_per_site": float(st[0].item()) / N}

    tc = run("fp16", n)
    bpu = profiled_traffic_per_unit("fwd2d_tc_connected_52x52.md", "psr_fwd2d_tc.cu",
                                    "dram bytes per evaluated patch")
    conn_patches = tc["evaluated_patches_per_step"] - n * (Lx // 2) * (Ly // 2)
    pk, src = measured_peaks()
    peak = float(pk.get("bf16_tflops_sustained", pk.get("bf16_tflops")))
    f32 = run("fp32", min(n32, n))
    return {"model": "2D patched minGRU (2x2 patches, vertical h_V coupling), tcgen05 tensor cores "
                     "(FP16 operands, FP32 accumulation, gates, scan, softmax)",
            "lattice": f"{Lx}x{Ly} OBC", "hidden": H, "layers": N_LAYERS, "samples": n,
            "connected": tc["connected"], "value": tc["value"], "unit": UNIT, "ms_per_step": tc["ms_per_step"],
            "evaluated_patches_per_step": tc["evaluated_patches_per_step"],
            "energy_per_site": tc["energy_per_site"],
            "roofline": {"kernel": "fwd2d_tc_kernel (connected configurations)", "bound": "tensor",
                         "achieved": tc["achieved_tflops"], "peak": peak, "unit": "TFLOP/s",
                         "frac": tc["achieved_tflops"] / peak,
                         "peak_source": f"{src} dense BF16 tensor rate, sustained (FP16 runs at the same rate)",
                         "traffic": (bpu * conn_patches) if bpu is not None else None,
                         "traffic_source": "DRAM bytes per evaluated patch of the committed ncu "
                                           "summary (4-sample capture) x the launch's evaluated patches",
                         "flops_per_unit": flops_per_patch_2d(H),
                         "launch_ms": tc["connected_launch_ms"]},
            "fp32_cuda_cores": {"samples": f32["samples"], "value": f32["value"], "unit": UNIT,
                                "ms_per_step": f32["ms_per_step"], "achieved_tflops": f32["achieved_tflops"],
                                "frac_of_fp32_simt_peak": f32["achieved_tflops"] / FP32_SIMT_TFLOPS,
                                "energy_per_site": f32["energy_per_site"]},
            "speedup_vs_fp32": tc["value"] / f32["value"]}


# FLOPs per evaluated site of the deep LRU (3 layers, hidden H): layer 0:
# Re(C h) and the two GLU products (2 x 2H^2 + 2 x 2H^2); layers 1, 2: also
# the complex B u (2 x 2H^2), so 12 H^2 each.
def lru_flops_per_site(H):
    return 8 * H * H + 2 * 12 * H * H


def lru_leg(dev, N=256, H=64, n=1024, reps=3):
    """The paper's deep 1D LRU on the 1D TFIM (Table IV configuration: 3
    layers, d = d_h = 64, N = 256 OBC, 1024 samples, h = 1): log psi + E_loc
    over every site flip on the tensor cores (FP16 operands, FP32
    accumulation, complex scan, GLU and readout) and on the FP32 CUDA cores;
    then the gradient's reverse pass, the exact sampler, and one full VMC
    step (sampling, E_loc, gradient, Adam) at both precisions (at FP16 the
    sampler and E_loc run on the tensor cores, the gradient in FP32)."""
    import torch

    from paper_2605_13807_gb300 import api, binding as B, inputs
    ham = B.make_hamiltonian("tfim", N, 1, False, True, 1.0, 1.0)
    theta = torch.from_numpy(inputs.lru_params(N_LAYERS, H, seed=0)).to(dev)
    spins = torch.from_numpy(inputs.random_spins(2000, n, N)).to(dev)
    lp = torch.empty(n, dtype=torch.float32, device=dev)
    el = torch.empty(n, dtype=torch.float32, device=dev)
    st = torch.empty(3, dtype=torch.float64, device=dev)
    E = n * N
    ctx = B.context()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    # sites evaluated by the connected forward: each flip at p resumes at its chunk
    p = torch.arange(N, device=dev)
    conn_sites = n * int((N - (p // 32) * 32).sum().item())

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    def run(prec):
        cfg = api.ModelConfig(N_LAYERS, H, False, prec)

        def step():
            api.logpsi_lru(theta, spins, cfg, out=lp)
            api.local_energy_lru(theta, spins, cfg, ham, out=el, stats=st)

        ms = timed(step)
        B.psr_context_set_profiling(ctx, True)
        api.local_energy_lru(theta, spins, cfg, ham, out=el, stats=st)
        conn_ms = B.psr_context_stage_ms(ctx)["fwd_connected"]
        B.psr_context_set_profiling(ctx, False)
        achieved = conn_sites * lru_flops_per_site(H) / (conn_ms / 1e3) / 1e12
        g = torch.Generator(device=dev)
        g.manual_seed(6)
        u = torch.rand((n, N), generator=g, device=dev)
        adam = api.Adam(theta.numel(), dev, lr=1e-3)
        th = theta.clone()  # updated in place by every step
        out = {}

        def vmc():
            out.update(api.vmc_step_lru(th, cfg, ham, u, adam, theta_out=th))

        vmc_ms = timed(vmc)
        # the exact sampler alone (1024 samples of the chain)
        sample_ms = timed(lambda: api.sample_lru(theta, u, cfg))
        # the same step at shorter chains, beside the paper's Table I step
        # times (1x H100, same model and sample count; context, not a target)
        by_n = {}
        for Nc in (32, 64, 128):
            ham_c = B.make_hamiltonian("tfim", Nc, 1, False, True, 1.0, 1.0)
            u_c = torch.rand((n, Nc), generator=g, device=dev)
            th_c = theta.clone()
            adam_c = api.Adam(theta.numel(), dev, lr=1e-3)
            by_n[str(Nc)] = timed(lambda: api.vmc_step_lru(th_c, cfg, ham_c, u_c, adam_c, theta_out=th_c))
        by_n[str(N)] = vmc_ms
        return {"value": (n + E) * N / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
                "connected_launch_ms": conn_ms, "achieved_tflops": achieved,
                "energy_per_site": float(st[0].item()) / N, "vmc_step_ms": vmc_ms, "sample_ms": sample_ms,
                "vmc_step_ms_by_N": by_n, "vmc_energy_per_site": float(out["stats"][0].item()) / N}

    tc = run("fp16")
    f32 = run("fp32")
    # reverse-mode gradient (dout-weighted sum), FP32
    w = torch.full((n,), 1.0 / n, dtype=torch.float32, device=dev)
    B.psr_context_set_profiling(ctx, True)
    api.grad_lru(theta, spins, api.ModelConfig(N_LAYERS, H, False, "fp32"), dout=w)
    bwd_ms = B.psr_context_stage_ms(ctx)["bwd"]
    B.psr_context_set_profiling(ctx, False)
    bpu = profiled_traffic_per_unit("lru_tc_connected_tfim256.md", "psr_lru_tc.cu",
                                    "dram bytes per evaluated site")
    pk, src = measured_peaks()
    peak = float(pk.get("bf16_tflops_sustained", pk.get("bf16_tflops")))
    return {"model": "deep 1D LRU (complex diagonal recurrence + GLU), tcgen05 tensor cores "
                     "(FP16 operands, FP32 accumulation, complex scan, GLU, readout)",
            "grad_bwd_ms": bwd_ms, "vmc_step_ms": tc["vmc_step_ms"], "vmc_step_ms_by_N": tc["vmc_step_ms_by_N"],
            "sample_ms": tc["sample_ms"],
            "paper_step_ms_H100_by_N": {"32": 28, "64": 71, "128": 260, "256": 900},
            "vmc_energy_per_site": tc["vmc_energy_per_site"],
            "workload": f"tfim_chain_{N}_obc_{n}_samples", "hidden": H, "connected": E,
            "value": tc["value"], "unit": UNIT, "ms_per_step": tc["ms_per_step"],
            "energy_per_site": tc["energy_per_site"],
            "roofline": {"kernel": "lru_tc_kernel (connected configurations)", "bound": "tensor",
                         "achieved": tc["achieved_tflops"], "peak": peak, "unit": "TFLOP/s",
                         "frac": tc["achieved_tflops"] / peak,
                         "peak_source": f"{src} dense BF16 tensor rate, sustained (FP16 runs at the same rate)",
                         "traffic": (bpu * conn_sites) if bpu is not None else None,
                         "traffic_source": "DRAM bytes per evaluated site of the committed ncu summary "
                                           "x the launch's evaluated sites",
                         "flops_per_unit": lru_flops_per_site(H), "launch_ms": tc["connected_launch_ms"]},
            "fp32_cuda_cores": {"value": f32["value"], "unit": UNIT, "ms_per_step": f32["ms_per_step"],
                                "connected_launch_ms": f32["connected_launch_ms"],
                                "achieved_tflops": f32["achieved_tflops"],
                                "frac_of_fp32_simt_peak": f32["achieved_tflops"] / FP32_SIMT_TFLOPS,
                                "energy_per_site": f32["energy_per_site"],
                                "vmc_step_ms": f32["vmc_step_ms"], "vmc_step_ms_by_N": f32["vmc_step_ms_by_N"],
                                "sample_ms": f32["sample_ms"],
                                "vmc_energy_per_site": f32["vmc_energy_per_site"]},
            "speedup_vs_fp32": tc["value"] / f32["value"]}


# The mixed persistent batch: 2D Heisenberg 16x16, 24x24, 32x32 (open, zero
# magnetisation, Neel-like samples) and the 2D TFIM 20x20 at h/J = 3.044
# (open, uniform random spins), 2048 samples each, hidden 128, BF16.
MIXED_SPEC = (("heisenberg", 16, True, 0.0), ("heisenberg", 24, True, 0.0),
              ("heisenberg", 32, True, 0.0), ("tfim", 20, False, 3.044))


def mixed_leg(dev, n=2048, reps=3, warmup=2):
    """One hot-path step (log psi, per-sample O_k and E_loc over every
    connected configuration) of four sample sets on different lattices and
    Hamiltonians in one psr_step_batch call: one launch per kernel of the
    step over all lattices, the forward shape picked by the autotuner on the
    first call, the launch sequence captured in a CUDA graph on the next and
    replayed in the timed steps."""
    import torch

    from paper_2605_13807_gb300 import api, binding as B, inputs
    theta = torch.from_numpy(inputs.glorot_params(N_LAYERS, HIDDEN, seed=0)).to(dev)
    P = theta.numel()
    items, logical, evaluated_conn, evaluated = [], 0, 0, 0
    for k, (kind, L, u1, hf) in enumerate(MIXED_SPEC):
        N = L * L
        s = (inputs.neel_like_spins(3000 + k, n, L, L) if kind == "heisenberg"
             else inputs.random_spins(3000 + k, n, N))
        sp = torch.from_numpy(s).to(dev)
        ham = B.make_hamiltonian(kind, L, L, False, True, 1.0, hf)
        _, ent, _ = api.connected(sp, ham)
        E = int(ent.shape[0])
        p = ent[:, 1].to(torch.int64)
        conn = int((N - (p // CHUNK_BF16) * CHUNK_BF16).sum().item())
        logical += (n + E) * N
        evaluated_conn += conn
        evaluated += n * N + conn
        out = {"logpsi": torch.empty(n, dtype=torch.float32, device=dev),
               "eloc": torch.empty(n, dtype=torch.float32, device=dev),
               "stats": torch.empty(3, dtype=torch.float64, device=dev),
               "grad": torch.empty((n, P), dtype=torch.float32, device=dev)}
        items.append((sp, ham, u1, out, E, f"{kind}_{L}x{L}"))
        del ent, p
    stream = torch.cuda.Stream(device=dev)
    ctx = B.context(stream)
    p_ = B.make_params(theta, N_LAYERS, HIDDEN, False, "bf16", ctx)
    args = [(sp, ham, u1, o["logpsi"], o["eloc"], o["stats"], o["grad"]) for sp, ham, u1, o, _, _ in items]
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        # uncaptured call with the tuner on (picks the forward shape of this
        # batch) and per-stage events (connected-forward time for the roofline)
        B.psr_context_set_autotune(ctx, True)
        B.psr_step_batch(p_, args)
        B.psr_context_set_autotune(ctx, False)
        B.psr_context_set_profiling(ctx, True)
        B.psr_step_batch(p_, args)
        stages = B.psr_context_stage_ms(ctx)
        B.psr_context_set_profiling(ctx, False)
        B.psr_context_set_graphs(ctx, True)
        for _ in range(warmup):           # capture, then replays
            B.psr_step_batch(p_, args)
        B.psr_context_sync(ctx)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            B.psr_step_batch(p_, args)
        e1.record(stream)
        e1.synchronize()
        B.psr_context_sync(ctx)
        B.psr_context_set_graphs(ctx, False)
    ms = e0.elapsed_time(e1) / reps
    conn_ms = stages["fwd_connected"]
    peaks, peak_src = measured_peaks()
    peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops")))
    achieved = evaluated_conn * MMA_FLOPS_PER_SITE / (conn_ms / 1e3) / 1e12
    res = {"workload": "mixed batch: heisenberg 16x16, 24x24, 32x32 OBC + tfim 20x20 OBC h/J=3.044, "
                       f"{n} samples each, hidden 128, BF16",
           "call": "psr_step_batch (log psi + O_k + E_loc), CUDA-graph replay",
           "value": logical / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
           "logical_units_per_step": logical, "evaluated_units_per_step": evaluated,
           "stages_ms_uncaptured": stages,
           "items": {name: {"connected": E, "mean_energy_per_site": float(o["stats"][0].item()) / (h.Lx * h.Ly)}
                     for _, h, _, o, E, name in items},
           "roofline": {"kernel": "fwd_bf16_kernel (connected configurations of all four lattices, one launch)",
                        "bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                        "frac": achieved / peak, "peak_source": f"bf16_tflops_sustained of {peak_src}",
                        "traffic": None, "launch_ms": conn_ms, "units_per_launch": evaluated_conn,
                        "flops_per_unit": MMA_FLOPS_PER_SITE}}
    shape, tuned = B.psr_fwd_shape_for(ctx, "bf16", 2, [n] * len(MIXED_SPEC),
                                       [L * L for _, L, _, _ in MIXED_SPEC])
    res["bf16_seqs_per_mma_stream"] = {"shape": shape, "tuned": tuned}
    del items, args
    torch.cuda.empty_cache()
    return res


def vmc_leg(dev, L=10, n=1024, reps=3):
    """One full on-device VMC step (exact sampling, E_loc, energy gradient,
    Adam; the paper's definition of a training step, Sec. III.A) for the
    chain model on the 10x10 Heisenberg lattice (hidden 128, 3 layers, BF16
    sampling and E_loc on the tensor cores, FP32 gradient), without and with c4v
    symmetrisation (8 images per configuration)."""
    import torch

    from paper_2605_13807_gb300 import api, binding as B, inputs
    N = L * L
    ham = B.make_hamiltonian("heisenberg", L, L, False, True, 1.0, 0.0)
    cfg = api.ModelConfig(N_LAYERS, HIDDEN, True, "bf16")
    theta = torch.from_numpy(inputs.glorot_params(N_LAYERS, HIDDEN, seed=0)).to(dev)
    g = torch.Generator(device=dev)
    g.manual_seed(5)
    u = torch.rand((n, N), generator=g, device=dev)
    us = torch.rand(n, generator=g, device=dev)
    res = {"workload": f"heisenberg_{L}x{L}_obc_{n}_samples", "hidden": HIDDEN,
           "layers": N_LAYERS, "precision": "BF16 sampling and E_loc (tensor cores), FP32 gradient"}
    for sym in (False, True):
        adam = api.Adam(theta.numel(), dev, lr=1e-3)
        th = theta.clone()  # updated in place by every step
        out = api.vmc_step(th, cfg, ham, u, adam, symmetrize=sym, sym_uniforms=us, theta_out=th)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            out = api.vmc_step(th, cfg, ham, u, adam, symmetrize=sym, sym_uniforms=us, theta_out=th)
        e1.record()
        e1.synchronize()
        key = "c4v" if sym else "plain"
        res[key] = {"ms_per_step": e0.elapsed_time(e1) / reps,
                    "energy_per_site": float(out["stats"][0].item()) / N}
    # the paper's 2D patched minGRU (hidden 128 here: its gradient kernel
    # keeps a row's tiles in shared memory up to that width)
    cfg2 = api.ModelConfig(N_LAYERS, HIDDEN, True, "fp16")
    th2 = torch.from_numpy(inputs.glorot_params2d(N_LAYERS, HIDDEN, seed=0)).to(dev)
    u2 = torch.rand((n, N // 4), generator=g, device=dev)
    adam = api.Adam(th2.numel(), dev, lr=1e-3)
    out = api.vmc_step2d(th2, cfg2, ham, u2, adam, theta_out=th2)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        out = api.vmc_step2d(th2, cfg2, ham, u2, adam, theta_out=th2)
    e1.record()
    e1.synchronize()
    res["model2d"] = {"ms_per_step": e0.elapsed_time(e1) / reps,
                      "precision": "FP16 tensor-core E_loc forward; FP32 sampling and gradient",
                      "energy_per_site": float(out["stats"][0].item()) / N}
    return res


# per-step wall times of the paper's 2D runs (Table VI, 1x A100 80GB, 3
# layers, d_h = 256, 2x2 patches, c4v, 200 samples): context, not a target
PAPER_2D_STEP_S = {10: 0.5, 20: 8.2, 52: 405.6}


def paper2d_leg(dev, sizes=(10, 20), n=200, reps=2, warmup=1):
    """One on-device VMC step of the 2D patched minGRU at the paper's 2D
    configuration (3 layers, d_h = 256, 2x2 patches, c4v symmetrisation,
    200 samples, Heisenberg OBC with zero magnetisation): exact sampling,
    symmetrised E_loc (8 images; the tensor-core forward, FP16 operands), the
    gradient over the 8 images, Adam (sampling and gradient FP32 CUDA cores)."""
    import torch

    from paper_2605_13807_gb300 import api, binding as B, inputs
    H = 256
    cfg = api.ModelConfig(N_LAYERS, H, True, "fp16")
    res = {"model": "2D patched minGRU, c4v-symmetrised VMC step", "hidden": H, "layers": N_LAYERS,
           "samples": n, "precision": "FP16 tensor-core E_loc forward; FP32 sampling, image weights, gradient",
           "paper_step_s_A100": {}}
    g = torch.Generator(device=dev)
    g.manual_seed(7)
    for L in sizes:
        ham = B.make_hamiltonian("heisenberg", L, L, False, True, 1.0, 0.0)
        th = torch.from_numpy(inputs.glorot_params2d(N_LAYERS, H, seed=0)).to(dev)
        u = torch.rand((n, (L // 2) ** 2), generator=g, device=dev)
        us = torch.rand(n, generator=g, device=dev)
        adam = api.Adam(th.numel(), dev, lr=1e-3)
        api.sample2d(th, u, cfg, L, L)  # the sampler's tile is tuned here, outside the timing
        for _ in range(warmup):
            api.vmc_step2d(th, cfg, ham, u, adam, theta_out=th, symmetrize=True, sym_uniforms=us)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            out = api.vmc_step2d(th, cfg, ham, u, adam, theta_out=th, symmetrize=True, sym_uniforms=us)
        e1.record()
        e1.synchronize()
        res[f"{L}x{L}"] = {"ms_per_step": e0.elapsed_time(e1) / reps,
                           "energy_per_site": float(out["stats"][0].item()) / (L * L)}
        if L in PAPER_2D_STEP_S:
            res["paper_step_s_A100"][f"{L}x{L}"] = PAPER_2D_STEP_S[L]
    return res


def paper2d_sizes(args):
    return tuple(int(x) for x in args.paper2d_sizes.split(",") if x)


def run_model2d_only(args):
    import torch

    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    res = model2d_leg(52, 52, args.samples_2d, torch.device("cuda", 0))
    print(json.dumps({"model2d": res}), flush=True)
    return 0


def run_lru_only(args):
    import torch

    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    print(json.dumps({"lru": lru_leg(torch.device("cuda", 0), n=args.samples_lru)}), flush=True)
    return 0


def run_paper2d_only(args):
    import torch

    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    res = paper2d_leg(torch.device("cuda", 0), sizes=paper2d_sizes(args), reps=args.paper2d_reps,
                      warmup=args.paper2d_warmup)
    print(json.dumps({"paper2d_vmc_step": res}), flush=True)
    return 0


def run_mixed_only(args):
    import torch

    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    print(json.dumps({"mixed_batch": mixed_leg(torch.device("cuda", 0))}), flush=True)
    return 0


def depth_leg(dev, L=52, ns=(1, 16, 200, 4096), reps=5):
    """Where the fused forward's sequential-in-chunk recurrence stops being
    the right choice: log psi of n samples at L x L (BF16, one launch, no
    connected configurations) for small and large n, beside one standalone
    parallel scan (psr_scan: warp-shuffle step scans with a decoupled
    look-back carry between chunks) of one layer of the same n sequences of
    L^2 sites x 128 units, the kernel a scan-based evaluation of the
    recurrence would run three times per forward."""
    import torch

    from paper_2605_13807_gb300 import api, binding as B, inputs
    ctx = B.context()
    B.psr_context_set_profiling(ctx, True)
    N = L * L
    theta = torch.from_numpy(inputs.glorot_params(N_LAYERS, HIDDEN, seed=0)).to(dev)
    cfg = api.ModelConfig(N_LAYERS, HIDDEN, True, "bf16")
    out = {}
    for n in ns:
        sp = torch.from_numpy(inputs.neel_like_spins(4000 + n, n, L, L)).to(dev)
        lp = torch.empty(n, dtype=torch.float32, device=dev)
        api.logpsi(theta, sp, cfg, out=lp)
        fwd = []
        for _ in range(reps):
            api.logpsi(theta, sp, cfg, out=lp)
            fwd.append(B.psr_context_stage_ms(ctx)["fwd_samples"])
        a, b, h0 = inputs.scan_inputs_device(7, n, N, HIDDEN, dev)
        h = torch.empty_like(a)
        B.psr_context_set_autotune(ctx, True)
        api.scan(a, b, h0, out=h)
        B.psr_context_set_autotune(ctx, False)
        sc = []
        for _ in range(reps):
            api.scan(a, b, h0, out=h)
            sc.append(B.psr_context_stage_ms(ctx)["scan"])
        tile, _ = B.psr_scan_tile_for(ctx, n, N, HIDDEN)
        out[str(n)] = {"fused_forward_ms": min(fwd), "scan_one_layer_ms": min(sc),
                       "scan_tile": {"units": tile[0], "chunk": tile[1]},
                       "fused_sites_per_us": n * N / (min(fwd) * 1e3)}
        del a, b, h0, h, sp, lp
        torch.cuda.empty_cache()
    B.psr_context_set_profiling(ctx, False)
    return {"lattice": f"{L}x{L}", "hidden": HIDDEN, "by_samples": out}


def run_depth_only(args):
    import torch

    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    print(json.dumps({"depth": depth_leg(torch.device("cuda", 0))}), flush=True)
    return 0


def run_sample_only(args):
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2605_13807_gb300 import inputs
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    Lx, Ly, n = WORKLOADS[args.workload]
    n = args.sample_n or n
    theta = torch.from_numpy(inputs.glorot_params(N_LAYERS, HIDDEN, seed=0)).to(dev)
    print(json.dumps({"sample": sample_leg(theta, n, Lx * Ly, dev)}), flush=True)
    return 0


def run_scan_only(args):
    import torch

    import __graft_entry__
    __graft_entry__.build()
    Lx, Ly, n = WORKLOADS[args.workload]
    n = args.scan_n or n
    torch.cuda.set_device(0)
    print(json.dumps({"scan": scan_leg(args, n, Lx * Ly, torch.device("cuda", 0))}), flush=True)
    return 0


def run_mine(args):
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2605_13807_gb300 import api, binding as B, inputs

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    Lx, Ly, n = WORKLOADS[args.workload]
    N = Lx * Ly
    P = api.param_count(N_LAYERS, HIDDEN)
    ham = B.make_hamiltonian("heisenberg", Lx, Ly, False, True, 1.0, 0.0)
    cfg = api.ModelConfig(N_LAYERS, HIDDEN, True, "bf16")
    theta_np = inputs.glorot_params(N_LAYERS, HIDDEN, seed=0)
    spins_np = rank_samples(rank, n, Lx, Ly)
    theta = torch.from_numpy(theta_np).to(dev)
    spins = torch.from_numpy(spins_np).to(dev)
    lp = torch.empty(n, dtype=torch.float32, device=dev)
    el = torch.empty(n, dtype=torch.float32, device=dev)
    st = torch.empty(3, dtype=torch.float64, device=dev)
    ok = torch.empty((n, P), dtype=torch.float32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    # work accounting (untimed): connected set of these samples
    offs, ent, _ = api.connected(spins, ham)
    E = int(ent.shape[0])
    p = ent[:, 1].to(torch.int64)
    evaluated_conn = int((N - (p // CHUNK_BF16) * CHUNK_BF16).sum().item())
    logical = n * N + E * N
    evaluated = n * N + evaluated_conn
    del offs, ent, p

    ctx = B.context()
    B.psr_context_set_profiling(ctx, True)
    if args.fwd_shape:
        api.set_fwd_shape("bf16", args.fwd_shape)
    fwd_shape = api.fwd_shape_for("bf16", 1, n, N)[0]

    def step():
        api.logpsi(theta, spins, cfg, out=lp)
        api.grad(theta, spins, cfg, out=ok)
        api.local_energy(theta, spins, cfg, ham, out=el, stats=st)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        step()
    api.sync()

    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        gpu_id = str(local)
    clocks = Clocks(gpu_id)
    conn_ms, samp_ms = [], []
    total_ms = 0.0
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_wall = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        step()
        e1.record()
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        stages = B.psr_context_stage_ms(ctx)
        conn_ms.append(stages["fwd_connected"])
        samp_ms.append(stages["fwd_samples"])
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    api.sync()
    value, total_ms = whole_job_rate(logical * args.steps, total_ms, world, dev)
    ms_per_step = total_ms / args.steps
    evaluated_value, _ = whole_job_rate(evaluated * args.steps, total_ms, world, dev)

    # roofline of the dominant kernel: the connected-configuration forward
    peaks, peak_src = measured_peaks()
    conn_avg = sum(conn_ms) / len(conn_ms)
    flops = evaluated_conn * MMA_FLOPS_PER_SITE
    achieved = flops / (conn_avg / 1e3) / 1e12
    peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops")))
    tpu = profiled_traffic_per_unit()
    roofline = {"kernel": "fwd_bf16_kernel (connected configurations)", "bound": "tensor",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "peak_source": f"bf16_tflops_sustained of {peak_src}",
                "traffic": (tpu * evaluated_conn if tpu is not None else None),
                "algorithmic_flops_per_launch": flops, "launch_ms": conn_avg,
                "units_per_launch": evaluated_conn,
                "flops_per_unit": MMA_FLOPS_PER_SITE}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic (seeded Neel-like S^z=0 configurations, Glorot weights seed 0)",
        "config": {"workload": f"heisenberg_{Lx}x{Ly}_obc_{n}_samples", "lattice": f"{Lx}x{Ly} OBC",
                   "samples_per_gpu": n, "hidden": HIDDEN, "layers": N_LAYERS,
                   "precision": "BF16 tcgen05 projections, FP32 scan/softmax, FP32 backward",
                   "bf16_seqs_per_mma_stream": fwd_shape,
                   "connected_per_step": E, "logical_units_per_step": logical,
                   "evaluated_units_per_step": evaluated,
                   "l2": "256 MB buffer written between timed steps",
                   "parallelism": f"dp{world} (independent samples per GPU)"},
        "evaluated_value": evaluated_value,
        "roofline": roofline,
        "gpu_launches": args.steps * (sum(LAUNCHES.values()) + grad_launches(n, N)),
        "clocks": clk,
        "wall_s_timed_region": wall,
        "stages_ms_last_local_energy": B.psr_context_stage_ms(ctx),
    }

    # plain FP32 path on a bounded subset of the same samples
    if not args.no_fp32 and rank == 0:
        m = min(args.fp32_samples, n)
        cfg32 = api.ModelConfig(N_LAYERS, HIDDEN, True, "fp32")
        sub = spins[:m].contiguous()
        o2, e2 = api.connected(sub, ham)[:2]
        E2 = int(e2.shape[0])
        ok32 = torch.empty((m, P), dtype=torch.float32, device=dev)

        def step32():
            api.logpsi(theta, sub, cfg32, out=lp[:m])
            api.grad(theta, sub, cfg32, out=ok32)
            api.local_energy(theta, sub, cfg32, ham, out=el[:m], stats=st)

        step32()
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        reps32 = 3
        a0.record()
        for _ in range(reps32):
            step32()
        a1.record()
        a1.synchronize()
        ms32 = a0.elapsed_time(a1) / reps32
        line["fp32_path"] = {"value": (m * N + E2 * N) / (ms32 / 1e3), "unit": UNIT,
                             "samples": m, "ms": ms32, "repeats": reps32,
                             "note": "plain FP32 SIMT path, same workload on a sample subset; "
                                     "mean of 3 steps after one warm-up step"}
        del ok32

    if not args.no_scan and rank == 0:
        line["scan"] = scan_leg(args, n, N, dev)
    if not args.no_sample and rank == 0:
        line["sample"] = sample_leg(theta, n, N, dev)
    if not args.no_2d and rank == 0:
        line["model2d"] = model2d_leg(Lx, Ly, min(args.samples_2d, n), dev)
    if not args.no_lru and rank == 0:
        line["lru"] = lru_leg(dev, n=args.samples_lru)
    if not args.no_mixed and rank == 0:
        line["mixed_batch"] = mixed_leg(dev)
    if not args.no_vmc and rank == 0:
        line["vmc_step"] = vmc_leg(dev)
        line["paper2d_vmc_step"] = paper2d_leg(dev, sizes=paper2d_sizes(args), reps=args.paper2d_reps,
                                               warmup=args.paper2d_warmup)

    # end to end through the C ABI with host buffers
    if not args.no_e2e:
        sp_h = torch.from_numpy(spins_np).pin_memory()
        th_h = torch.from_numpy(theta_np).pin_memory()
        lp_h = torch.empty(n, dtype=torch.float32).pin_memory()
        el_h = torch.empty(n, dtype=torch.float32).pin_memory()
        st_h = torch.empty(3, dtype=torch.float64).pin_memory()
        ok_h = torch.empty((n, P), dtype=torch.float32).pin_memory()
        del ok
        torch.cuda.empty_cache()

        def step_host():
            api.logpsi(th_h, sp_h, cfg, out=lp_h)
            api.grad(th_h, sp_h, cfg, out=ok_h)
            api.local_energy(th_h, sp_h, cfg, ham, out=el_h, stats=st_h)

        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step_host()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e2e_value, e2e_ms = whole_job_rate(logical, dt * 1e3, world, dev)
        h2d = 3 * (n * N + P * 4)
        d2h = n * 4 + n * P * 4 + n * 4 + 3 * 8
        line["e2e"] = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms}

    if not args.no_cpu and world == 1 and rank == 0:
        v, cores, desc = oracle_rate(Lx, Ly, args.cpu_seconds / 1.0)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": desc}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.scan_only:
        return run_scan_only(args)
    if args.paper2d_only:
        return run_paper2d_only(args)
    if args.model2d_only:
        return run_model2d_only(args)
    if args.lru_only:
        return run_lru_only(args)
    if args.mixed_only:
        return run_mixed_only(args)
    if args.depth_only:
        return run_depth_only(args)
    if args.sample_only:
        return run_sample_only(args)
    return run_mine(args)


if __name__ == "__main__":
    sys.exit(main())
