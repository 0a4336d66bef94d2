#!/usr/bin/env python3
"""Throughput of the GB300 free-space Poisson solver (VGF and HE on the same GPU).

Workload (default): 3D VGF, 256^3 cells on [-1,1]^3, FP32, outputs phi and the
three components of E; rho = 8 seeded anisotropic Gaussians (centres
U[-0.5,0.5]^3, sigma_a U[0.05,0.15], Q U[-1,1], seed 1).  One step = one full
solve (all five passes).  HE is timed on the same GPU with the same input.
The working set (rho 67 MB, workspace 539 MB, outputs 268 MB) exceeds the
129 MB L2, so no flush is needed between iterations.

Multi-GPU: every rank solves its own replica (independent solves, no data-path
collective; weak scaling); the timing is the maximum over ranks.

--impl reference times the FP64 CPU oracle on this host instead: real 256^3
phi + E solves of the same problem, as many of the requested steps as fit in
about 150 s (the count timed is reported).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import platform
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "VGF free-space solves/s at 256^3 FP32 (phi+E), HE on the same GPU"
UNIT = "solves/s"


# ------------------------------------------------------------------ helpers

def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def pass_bytes(shape, with_E=True):
    """Algorithmic bytes per pass (FP32 real 4 B, complex 8 B).

    S = (n0+1) n1 n2 complex values: one half spectrum in k0 with n1 rows.
    P1 reads rho, writes S; P2 reads S, writes 2S; P3 reads 2S and the kernel
    octant, writes 2S per stream; P4 reads 2S per stream, writes S per output
    stream; P5 reads the output streams, writes the real outputs.
    """
    n0, n1, n2 = shape
    cells = n0 * n1 * n2
    S = (n0 + 1) * n1 * n2
    K = 4 * (n0 + 1) * (n1 + 1) * (n2 + 1)
    s3, s4, outs = (2, 3, 4) if with_E else (1, 1, 1)
    return {
        "p1_fwd": 4 * cells + 8 * S,
        "p2_fwd": 8 * S + 16 * S,
        "p3_fwd": 16 * S + K + s3 * 16 * S,
        "p4_fwd": s3 * 16 * S + s4 * 8 * S,
        "p5_fwd": s4 * 8 * S + 4 * outs * cells,
    }


def compulsory_bytes(shape, with_E=True):
    """Bytes no implementation can avoid: read rho and the kernel octant once, write the outputs once."""
    cells = int(np.prod(shape))
    outs = 1 + len(shape) if with_E else 1
    return 4 * cells + 4 * int(np.prod([n + 1 for n in shape])) + 4 * outs * cells


def pass_flops(shape, with_E=True):
    """FP32 flops of the transforms per pass, by the usual count: 5 L log2 L per complex line of length L,
    half that per real line, padded lengths, pruning ignored. 3D: R2C along axis 0 (n1 n2 real lines),
    forward along axis 1 (H n2 lines, H = n0+1), along axis 2 (H 2n1 lines: one forward, one inverse
    per stream), inverse along axis 1 (H n2 lines per output stream), one C2R per real output.
    2D: R2C, the fused pass (forward plus one inverse per stream), one C2R per real output."""
    def c(L):
        return 5 * L * math.log2(L)
    if len(shape) == 3:
        n0, n1, n2 = shape
        H = n0 + 1
        s3, s4, outs = (2, 3, 4) if with_E else (1, 1, 1)
        return {"p1_fwd": n1 * n2 * c(2 * n0) / 2, "p2_fwd": H * n2 * c(2 * n1),
                "p3_fwd": (1 + s3) * H * 2 * n1 * c(2 * n2), "p4_fwd": s4 * H * n2 * c(2 * n1),
                "p5_fwd": outs * n1 * n2 * c(2 * n0) / 2}
    n0, n2 = shape
    H = n0 + 1
    s3, outs = (2, 3) if with_E else (1, 1)
    return {"p1_fwd": n2 * c(2 * n0) / 2, "p3_fwd": (1 + s3) * H * c(2 * n2), "p5_fwd": outs * n2 * c(2 * n0) / 2}


def pipeline_flops(shape, with_E=True):
    return sum(pass_flops(shape, with_E).values())


def fp32_peak_tflops(sms, sm_mhz):
    """FP32 ALU peak from unit counts and clock: SMs x 128 FP32 lanes x 2 flops per FMA x SM clock."""
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


def device_sms(device=0):
    import torch
    return int(torch.cuda.get_device_properties(device).multi_processor_count)


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2103_08531_gb300", "csrc")
    for fn in sorted(os.listdir(csrc)):
        if fn.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(csrc, fn), "rb") as f:
                h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, workload):
    """dram read+write bytes per launch from a committed ncu summary, if still current."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        with open(path) as f:
            d = json.load(f)
        e = d.get(workload, {}).get(kernel)
        if e and e.get("source_hash") == kernel_source_hash():
            return int(e["dram_bytes"])
    except Exception:
        return None
    return None


def reduce_max(dist, x, device="cpu"):
    """Maximum of a per-rank scalar over all ranks (identity without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, world, max_ms):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / (max_ms * 1e-3)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------- CPU oracle

def oracle_sample(n=128, repeats=1):
    """Time the FP64 oracle's phi+E solve of the same mixture at n^3 (kernel precomputed)."""
    import oracle
    prob = W.mixture_3d(n, 8, 1)
    rho = prob.rho(np.float32).astype(np.float64)
    g = oracle.kernel_vgf(list(prob.shape), prob.h)
    times = []
    for _ in range(repeats):
        t = time.perf_counter()
        oracle.solve_with_kernel(g, rho, prob.h)
        times.append(time.perf_counter() - t)
    scale = (256 ** 3 * math.log2(512 ** 3)) / (n ** 3 * math.log2((2 * n) ** 3))
    return times, scale, oracle.threads()


def padded_fft_solve(octant, rho, h):
    """The solve with torch.fft on the unpruned padded grid (library context only):
    rfftn of rho zero-padded to 2n, times the kernel spectrum (octant[k] holds
    prod(h)/prod(2n) DFT(g)(k), mirrored to the other octants), one irfftn for phi
    and one per field component with -i k_a (Nyquist index zero), crop to n."""
    import torch
    n0, n1, n2 = rho.shape
    dev = rho.device
    N = (2 * n0, 2 * n1, 2 * n2)

    def fold(n, N_):
        k = torch.arange(N_, device=dev)
        return torch.where(k <= n, k, N_ - k)

    def wavek(n, N_, hh):
        k = torch.arange(N_, device=dev)
        m = torch.where(k < n, k, torch.where(k == n, torch.zeros_like(k), k - N_))
        return (2 * math.pi / (N_ * hh)) * m.to(rho.dtype)

    K = octant[fold(n0, N[0])][:, fold(n1, N[1])][:, :, : n2 + 1] * float(N[0] * N[1] * N[2])
    S = torch.fft.rfftn(rho, s=N) * K   # irfftn divides by prod(2n) again
    ws = (wavek(n0, N[0], h[0])[:, None, None], wavek(n1, N[1], h[1])[None, :, None],
          wavek(n2, N[2], h[2])[None, None, : n2 + 1])
    phi = torch.fft.irfftn(S, s=N)[:n0, :n1, :n2]
    E = [torch.fft.irfftn(S * (-1j * w), s=N)[:n0, :n1, :n2] for w in ws]
    return phi, E


def cufft_context(plan, rho, phi, E, steps=20, warmup=3):
    """Context only (a library baseline, not the product path): padded_fft_solve
    on the GPU (cuFFT through torch.fft) for the same problem; its time per solve
    and its agreement with our solve."""
    import torch
    octant = torch.from_numpy(plan.kernel_spectrum()).to(rho.device)
    plan.solve(rho, phi=phi, E=E)
    for _ in range(warmup):
        p_c, E_c = padded_fft_solve(octant, rho, plan.h)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        p_c, E_c = padded_fft_solve(octant, rho, plan.h)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    err_phi = float((p_c - phi).abs().max() / phi.abs().max())
    err_E = float((torch.stack(E_c) - E).abs().max() / E.abs().max())
    return {"kind": "library context (torch.fft / cuFFT), not the product path",
            "what": "rfftn of rho zero-padded to 2n, times the same kernel spectrum (and -i k_a), "
                    "one irfftn per output, crop; unpruned",
            "ms_per_step": ms, "solves_per_s": 1e3 / ms, "max_rel_diff_phi": err_phi, "max_rel_diff_E": err_E}


def torch_cpu_context(n=128):
    """Context only: padded_fft_solve with torch.fft on the host cores (FP32) at n^3,
    scaled to 256^3 by the N^3 log N work ratio."""
    import torch
    prob = W.mixture_3d(n, 8, 1)
    import oracle
    g = oracle.kernel_vgf(list(prob.shape), prob.h)
    octant = torch.from_numpy(oracle.scaled_spectrum_octant(g, prob.h)).to(torch.float32)
    rho = torch.from_numpy(prob.rho(np.float32))
    padded_fft_solve(octant, rho, prob.h)
    t = time.perf_counter()
    padded_fft_solve(octant, rho, prob.h)
    t = time.perf_counter() - t
    scale = (256 ** 3 * math.log2(512 ** 3)) / (n ** 3 * math.log2((2 * n) ** 3))
    return {"kind": "library context (torch.fft on the host cores, FP32), not the product path",
            "threads": torch.get_num_threads(), "sample": f"one solve at {n}^3 ({t:.2f} s), scaled by {scale:.2f}",
            "solves_per_s": 1.0 / (t * scale)}


def cpu_model() -> str:
    """The host CPU's name as the kernel reports it (x86 'model name', else the Arm part number)."""
    try:
        info = open("/proc/cpuinfo").read().splitlines()
    except OSError:
        return platform.processor() or "unknown"
    arm_parts = {"0xd4f": "Arm Neoverse-V2", "0xd40": "Arm Neoverse-V1", "0xd0c": "Arm Neoverse-N1",
                 "0xd49": "Arm Neoverse-N2"}
    for key in ("model name", "Model Name", "CPU part"):
        for line in info:
            if line.startswith(key):
                val = line.split(":", 1)[1].strip()
                return arm_parts.get(val, f"{key}: {val}")
    return platform.machine()


def oracle_headline(repeats=1, budget_s=None, n=256):
    """Time the FP64 oracle's phi+E solve of the headline problem itself (256^3, 8 anisotropic
    Gaussians, seed 1), kernel precomputed outside the timing (as the GPU plan is).  Runs `repeats`
    solves, or fewer once `budget_s` seconds of solving have passed (at least one)."""
    import oracle
    prob = W.mixture_3d(n, 8, 1)
    rho = prob.rho(np.float32).astype(np.float64)
    g = oracle.kernel_vgf(list(prob.shape), prob.h)
    times = []
    for _ in range(repeats):
        t = time.perf_counter()
        oracle.solve_with_kernel(g, rho, prob.h)
        times.append(time.perf_counter() - t)
        if budget_s is not None and sum(times) >= budget_s:
            break
    return times, oracle.threads()


def cpu_baseline_block(n=128, n1=64, full_n=256):
    """The oracle on all host threads: one real solve of the headline workload at 256^3 (the
    figure), plus two labelled extras scaled from smaller samples by the N^3 log N work ratio:
    all threads at n^3, one thread at n1^3."""
    import oracle
    t_full, cores = oracle_headline(1, n=full_n)
    t = t_full[0]
    times, scale, _ = oracle_sample(n)
    ts = min(times)
    prev = oracle.threads()
    oracle.set_threads(1)
    try:
        t1s, scale1, _ = oracle_sample(n1)
    finally:
        oracle.set_threads(prev)
    t1 = min(t1s)
    return {"value": 1.0 / t, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"one FP64 oracle phi+E solve of the headline workload itself ({full_n}^3, 8-Gaussian "
                      f"mixture, seed 1): {t:.2f} s; the VGF kernel is precomputed outside the timing",
            "cpu": cpu_model(),
            "scaled_sample": {"value": 1.0 / (ts * scale), "unit": UNIT, "cores": cores,
                              "sample": f"the same mixture at {n}^3 ({ts:.2f} s), scaled to 256^3 by the N^3 log N "
                                        f"work ratio {scale:.2f} (an extrapolation, for comparison only)"},
            "single_thread": {"value": 1.0 / (t1 * scale1), "unit": UNIT, "cores": 1,
                              "sample": f"the same mixture at {n1}^3 on one thread ({t1:.2f} s), "
                                        f"scaled by {scale1:.2f} (an extrapolation)"}}


def run_reference(args, budget_s=150.0):
    """The reference arm: the FP64 oracle on the host cores, real 256^3 solves of the headline
    workload.  Warm-up steps are small (64^3) solves; the timed steps are full solves, as many of the
    requested ones as fit in about `budget_s` seconds (at least one), and the line reports the count
    actually timed."""
    ws, rank, _ = dist_info()
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        oracle_sample(64)
    times, cores = oracle_headline(args.steps, budget_s)
    total = sum(times)
    k = len(times)
    value = k / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": k, "steps_requested": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * total / k,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": "3D VGF 256^3 on [-1,1]^3, 8 anisotropic Gaussians (seed 1), "
                                                        "phi+E; FP64 oracle on the host cores"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{k} FP64 oracle phi+E solves of the headline workload at 256^3 "
                                       f"({total:.1f} s; kernel precomputed outside the timing; warm-up steps are "
                                       f"64^3 solves; timed steps capped at about {budget_s:.0f} s)",
                             "cpu": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- GPU arm

def run_gpu(args):
    import torch
    ws, rank, local = dist_info()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist_mod
        dist_mod.init_process_group("nccl" if torch.distributed.is_nccl_available() else "gloo")
        dist = dist_mod
    import paper_2103_08531_gb300 as fsp
    from paper_2103_08531_gb300 import build
    build.build()

    prob = W.mixture_3d(256, 8, 1)
    rho_host = torch.from_numpy(prob.rho(np.float32)).pin_memory()
    rho = rho_host.to(f"cuda:{local}")
    plan_s = {}
    plans = {}
    for m in ("vgf", "he"):
        t = time.perf_counter()
        plans[m] = fsp.Plan(prob.shape, prob.h, m)
        plan_s[m] = time.perf_counter() - t
    tuning = load_tuning(plans["vgf"], prob.shape)
    phi = torch.empty_like(rho)
    E = torch.empty((3,) + prob.shape, dtype=torch.float32, device=rho.device)
    stream = torch.cuda.current_stream()
    npass = 5

    def barrier():
        if dist is not None:
            dist.barrier()

    def reduce_max_local(x):
        return reduce_max(dist, x, rho.device if dist is not None and dist.get_backend() == "nccl" else "cpu")

    for m in ("vgf", "he"):
        for _ in range(args.warmup):
            plans[m].solve(rho, phi=phi, E=E)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    results = {}
    for m in ("vgf", "he"):
        plan = plans[m]
        # (1) the headline: K back-to-back solves, nothing recorded between the
        # passes (an event between two passes would stop the next pass from
        # being scheduled while the previous one finishes)
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        start.record(stream)
        for s in range(args.steps):
            plan.solve(rho, phi=phi, E=E)
        end.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = start.elapsed_time(end)
        # (2) per-pass split: the same K solves again with an event at every pass boundary
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(npass + 1)] for _ in range(args.steps)]
        for row in evs:
            for e in row:
                e.record(stream)
        torch.cuda.synchronize()
        for s in range(args.steps):
            plan.set_pass_events(evs[s])
            plan.solve(rho, phi=phi, E=E)
        torch.cuda.synchronize()
        plan.set_pass_events(None)
        per_pass = [statistics.mean(evs[s][i].elapsed_time(evs[s][i + 1]) for s in range(args.steps))
                    for i in range(npass)]
        results[m] = {"ms": reduce_max_local(ms), "per_pass_ms": per_pass,
                      "ms_with_pass_events": sum(per_pass)}
    clk = clocks.stop()

    # end to end through the C ABI's host pipe (fsp_host_pipe_solve): pinned host rho in, phi and E
    # back to pinned host memory every step; copy-in, solve and copy-out on the library's three
    # streams, so the transfers of neighbouring solves overlap.  W warm-up solves through the same
    # pipe first.
    e2e_ms = None
    if not args.no_e2e:
        pipe = fsp.HostPipeline(plans["vgf"], depth=2)
        phis_h = [torch.empty(prob.shape, dtype=torch.float32).pin_memory() for _ in range(2)]
        Es_h = [torch.empty((3,) + prob.shape, dtype=torch.float32).pin_memory() for _ in range(2)]
        pipe.run([rho_host] * args.warmup, [phis_h[i % 2] for i in range(args.warmup)],
                 [Es_h[i % 2] for i in range(args.warmup)], stream=stream)
        torch.cuda.synchronize()
        barrier()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        pipe.run([rho_host] * args.steps, [phis_h[i % 2] for i in range(args.steps)],
                 [Es_h[i % 2] for i in range(args.steps)], stream=stream)
        s1.record(stream)
        torch.cuda.synchronize()
        barrier()
        e2e_ms = reduce_max_local(s0.elapsed_time(s1))
        pipe.close()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    peak, peak_kind = measured_peaks()
    pb = pass_bytes(prob.shape, True)
    names = list(pb.keys())
    vgf = results["vgf"]
    dom = max(range(npass), key=lambda i: vgf["per_pass_ms"][i])
    dom_name = names[dom]
    achieved = pb[dom_name] / (vgf["per_pass_ms"][dom] * 1e-3) / 1e9
    total_bytes = sum(pb.values())
    ms_step = vgf["ms"] / args.steps
    value = job_value(args.steps, ws, vgf["ms"])
    he_ms_step = results["he"]["ms"] / args.steps
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "3D VGF 256^3 on [-1,1]^3, FP32, phi + E, 8 anisotropic Gaussians (seed 1)",
                   "grid": list(prob.shape), "method": "vgf", "outputs": "phi,Ex,Ey,Ez",
                   "l2": "working set 0.9 GB > 129 MB L2, no flush", "parallelism": f"replicas x{ws}"},
        "gpts_per_s": value * prob.points / 1e9,
        "he": {"ms_per_step": he_ms_step, "solves_per_s": ws / (he_ms_step * 1e-3),
               "per_pass_ms": results["he"]["per_pass_ms"]},
        "vgf_over_he_time": ms_step / he_ms_step,
        "plan_seconds": {"vgf": plan_s["vgf"], "he": plan_s["he"],
                         "what": "once per geometry, outside solves/s (FP64 kernel spectrum on the GPU)"},
        "per_pass_ms": dict(zip(names, vgf["per_pass_ms"])),
        "per_pass_note": "per-pass times from a second run of the same solves with an event at every pass "
                         "boundary (those events keep a pass from starting while the previous one finishes)",
        "ms_per_step_with_pass_events": vgf["ms_with_pass_events"],
        "per_pass_gbs": {k: pb[k] / (t * 1e-3) / 1e9 for k, t in zip(names, vgf["per_pass_ms"])},
        "pipeline": {"bytes": total_bytes, "gbs": total_bytes / (ms_step * 1e-3) / 1e9,
                     "frac": total_bytes / (ms_step * 1e-3) / 1e9 / peak},
        "compulsory": secondary_bytes(compulsory_bytes(prob.shape), ms_step, peak),
        "flops": secondary_flops(pipeline_flops(prob.shape), ms_step),
        "roofline": {"bound": "hbm", "kernel": dom_name, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind,
                     "traffic": ncu_traffic(dom_name, "vgf256"),
                     "algorithmic_bytes": pb[dom_name]},
        "alu_check": alu_check(dom_name, pass_flops(prob.shape)[dom_name], vgf["per_pass_ms"][dom],
                               device_sms(local), *alu_clock(clk)),
        "gpu_launches": npass * args.steps,
        "clocks": clk,
        "tuning": tuning,
    }
    if e2e_ms is not None:
        line["e2e"] = {"value": ws * args.steps / (e2e_ms * 1e-3), "unit": UNIT,
                       "h2d_bytes_per_step": rho.numel() * 4, "d2h_bytes_per_step": (phi.numel() + E.numel()) * 4,
                       "api": "fsp_host_pipe_solve (C ABI, pinned host buffers, 3 library streams, depth 2)"}
    if ws == 1 and not args.no_context:
        line["context"] = {"cufft": cufft_context(plans["vgf"], rho, phi, E)}
        if not args.no_cpu_baseline:
            line["context"]["torch_fft_cpu"] = torch_cpu_context()
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_block()
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


# ----------------------------------------------------------- other workloads

def pass_bytes_2d(shape, with_E=True):
    """Algorithmic bytes of the 2D pipeline (P1 axis 0 R2C, P3 fused along axis 1, P5 C2R)."""
    n0, n2 = shape
    cells = n0 * n2
    S = (n0 + 1) * n2
    K = 4 * (n0 + 1) * (n2 + 1)
    s3, outs = (2, 3) if with_E else (1, 1)
    return {"p1_fwd": 4 * cells + 8 * S, "p3_fwd": 8 * S + K + s3 * 8 * S, "p5_fwd": s3 * 8 * S + 4 * outs * cells}


def secondary_bytes(byts, ms, peak):
    return {"bytes": byts, "gbs": byts / (ms * 1e-3) / 1e9, "frac": byts / (ms * 1e-3) / 1e9 / peak,
            "what": "read rho and the kernel octant, write the outputs, once each"}


def secondary_flops(flops, ms):
    return {"per_solve": flops, "tflops": flops / (ms * 1e-3) / 1e12,
            "count": "5 L log2 L per complex line, half per real line, pruning ignored (FP32 ALU, not tensor)"}


def alu_check(kernel, flops, ms, sms, sm_mhz, clock_from):
    """The dominant kernel's transform arithmetic against the FP32 ALU peak (a secondary roofline):
    the peak counts this device's SMs at the SM clock sampled while the kernel ran."""
    tf = flops / (ms * 1e-3) / 1e12
    peak = fp32_peak_tflops(sms, sm_mhz)
    return {"kernel": kernel, "flops": flops, "tflops": tf, "peak_tflops": peak, "frac": tf / peak,
            "peak_from": f"{sms} SMs x 128 FP32 lanes x 2 (FMA) x {sm_mhz:.0f} MHz ({clock_from}); "
                         "flops by 5 L log2 L per line"}


def alu_clock(clk):
    """SM clock for the ALU peak: the median sampled under load, else the reported maximum, else 2070 MHz."""
    if clk and clk.get("sm_mhz"):
        return float(clk["sm_mhz"]), "median SM clock sampled in the timed region"
    if clk and clk.get("sm_max_mhz"):
        return float(clk["sm_max_mhz"]), "maximum SM clock reported by nvidia-smi"
    return 2070.0, "nominal maximum SM clock (no clock samples)"


def load_tuning(plan, shape):
    """Read the committed launch-variant cache (written by paper_2103_08531_gb300.tune on this GPU
    type) into the process-wide table; report the variants the plan's passes now use."""
    from paper_2103_08531_gb300 import tune as T
    import paper_2103_08531_gb300 as fsp
    have = os.path.exists(T.TUNE_CACHE)
    if have:
        plan.autotune(T.TUNE_CACHE, 0)
    lengths = {"p1_fwd": 2 * shape[0], "p3_fwd": 2 * shape[-1], "p5_fwd": 2 * shape[0]}
    if len(shape) == 3:
        lengths.update({"p2_fwd": 2 * shape[1], "p4_fwd": 2 * shape[1]})
    return {"cache": os.path.relpath(T.TUNE_CACHE, ROOT) if have else None,
            "variants": {f"{k}/{N}": fsp.tuned_variant(k, N) for k, N in sorted(lengths.items())}}


def _timed(fn, steps, warmup):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b)


def run_other(args):
    """Single-GPU measurements of the other workloads (one JSON line each)."""
    import torch
    import paper_2103_08531_gb300 as fsp
    from paper_2103_08531_gb300 import build
    build.build()
    peak, peak_kind = measured_peaks()
    clocks = ClockSampler(0)
    line = {"n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic"}
    if args.workload == "beam64":
        probs = W.beam_batch(64, seed=3)
        t = time.perf_counter()
        plans = [fsp.Plan(p.shape, p.h, "vgf") for p in probs]
        t_plan = time.perf_counter() - t
        line["tuning"] = load_tuning(plans[0], probs[0].shape)
        rhos = [torch.from_numpy(p.rho(np.float32)).cuda() for p in probs]
        batch = fsp.Batch(plans, rhos)
        kernels = batch.kernel_count()
        graph = batch.capture()
        clocks.start()
        ms = _timed(graph.replay, args.steps, args.warmup)
        ms_seq = _timed(lambda: [pl.solve(r, phi=ph, E=e) for pl, r, ph, e in
                                 zip(plans, rhos, batch.phis, batch.Es)], args.steps, args.warmup)
        clk = clocks.stop()
        pts = sum(p.points for p in probs)
        byts = sum(sum(pass_bytes(p.shape, True).values()) for p in probs)
        per = ms / args.steps
        line.update({"metric": "batched VGF solves/s, 64 uneven beam-bunch geometries, one graph replay per batch",
                     "value": 64 / (per * 1e-3), "unit": "solves/s", "ms_per_step": per,
                     "config": {"workload": "64 x 3D VGF, shapes from {64^3,96^3,128^3,64x64x256,128x128x512}, "
                                            "h_a U[0.005,0.03], one Gaussian each (seed 3), phi+E, CUDA graph"},
                     "gpts_per_s": pts / (per * 1e-3) / 1e9,
                     "pipeline": {"bytes": byts, "gbs": byts / (per * 1e-3) / 1e9,
                                  "frac": byts / (per * 1e-3) / 1e9 / peak, "peak_kind": peak_kind},
                     "sequential_ms_per_batch": ms_seq / args.steps, "plan_seconds_64_geometries": t_plan,
                     "kernels_per_batch": kernels, "gpu_launches": kernels * args.steps, "clocks": clk})
    elif args.workload == "gauss2d4096":
        prob = W.mixture_2d(4096, 16, 2)
        rho = torch.from_numpy(prob.rho(np.float32)).cuda()
        res = {}
        plan_s = {}
        clocks.start()
        per_pass = None
        for m in ("vgf", "he"):
            t = time.perf_counter()
            plan = fsp.Plan(prob.shape, prob.h, m)
            plan_s[m] = time.perf_counter() - t
            line["tuning"] = load_tuning(plan, prob.shape)
            phi = torch.empty_like(rho)
            E = torch.empty((2,) + prob.shape, device="cuda")
            res[m] = _timed(lambda: plan.solve(rho, phi=phi, E=E), args.steps, args.warmup) / args.steps
            if m == "vgf":
                evs = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
                for e in evs:
                    e.record()
                plan.set_pass_events(evs)
                plan.solve(rho, phi=phi, E=E)
                torch.cuda.synchronize()
                plan.set_pass_events(None)
                per_pass = dict(zip(["p1_fwd", "p3_fwd", "p5_fwd"], [evs[i].elapsed_time(evs[i + 1]) for i in range(3)]))
        clk = clocks.stop()
        byts = sum(pass_bytes_2d(prob.shape).values())
        per = res["vgf"]
        line.update({"metric": "2D VGF solves/s at 4096^2 FP32 (phi+E)", "value": 1e3 / per, "unit": "solves/s",
                     "ms_per_step": per, "config": {"workload": "2D VGF 4096^2 on [-1,1]^2, 16 Gaussians (seed 2)"},
                     "gpts_per_s": prob.points / (per * 1e-3) / 1e9, "he_ms_per_step": res["he"],
                     "per_pass_ms": per_pass,
                     "per_pass_gbs": {k: pass_bytes_2d(prob.shape)[k] / (t * 1e-3) / 1e9 for k, t in per_pass.items()},
                     "pipeline": {"bytes": byts, "gbs": byts / (per * 1e-3) / 1e9,
                                  "frac": byts / (per * 1e-3) / 1e9 / peak, "peak_kind": peak_kind},
                     "compulsory": secondary_bytes(compulsory_bytes(prob.shape), per, peak),
                     "flops": secondary_flops(pipeline_flops(prob.shape), per),
                     "plan_seconds": {"vgf": plan_s["vgf"], "he": plan_s["he"],
                                      "what": "once per geometry, outside solves/s"},
                     "gpu_launches": 3 * args.steps, "clocks": clk})
    elif args.workload == "train128":
        n, B = 128, 8
        probs, target = W.training_batch(n, B)
        plan = fsp.Plan((n, n, n), probs[0].h, "vgf")
        line["tuning"] = load_tuning(plan, (n, n, n))
        tgt = torch.from_numpy(target).cuda()
        rhos = [torch.from_numpy(p.rho(np.float32)).cuda().requires_grad_(True) for p in probs]

        def step():
            loss = 0.0
            for r in rhos:
                r.grad = None
                phi, E = fsp.FspSolve.apply(r, plan)
                loss = loss + ((phi - tgt) ** 2).sum() + 0.1 * (E ** 2).sum()
            loss.backward()

        clocks.start()
        per = _timed(step, args.steps, args.warmup) / args.steps
        clk = clocks.stop()
        line.update({"metric": "differentiable VGF: forward + adjoint per batch of 8 at 128^3 (loss on phi and E)",
                     "value": B / (per * 1e-3), "unit": "fwd+bwd items/s", "ms_per_step": per,
                     "config": {"workload": "8 x 128^3 VGF, 4-Gaussian densities (seeds 10..17), "
                                            "loss sum (phi - phi_t)^2 + 0.1 |E|^2"},
                     # five forward and five adjoint passes per item; torch's loss ops are not counted
                     "gpu_launches": 10 * B * args.steps, "clocks": clk})
    elif args.workload == "fd_direct":
        # the finite-difference field on a solved 256^3 HE potential, and FP64 direct-path solves at the
        # odd sizes of the paper's convergence studies
        prob = W.mixture_3d(256, 8, 1)
        plan = fsp.Plan(prob.shape, prob.h, "he")
        phi, _ = plan.solve(torch.from_numpy(prob.rho(np.float32)).cuda(), with_E=False)
        E = torch.empty((3,) + prob.shape, dtype=torch.float32, device="cuda")
        clocks.start()
        per_fd = _timed(lambda: plan.gradient_fd(phi, E), args.steps, args.warmup) / args.steps
        direct = {}
        for name, shape, h in (("13x17x11", (13, 17, 11), (0.05, 0.04, 0.06)), ("50x37", (50, 37), (0.02, 0.03))):
            d = len(shape)
            dp = fsp.Plan(shape, h, "vgf", dtype="f64")
            src = W.Problem(name, shape, h, [(np.zeros(d), np.full(d, 0.1), 1.0)])
            r = torch.from_numpy(src.rho(np.float64)).cuda()
            po = torch.empty_like(r)
            Eo = torch.empty((d,) + shape, dtype=torch.float64, device="cuda")
            direct[name] = _timed(lambda: dp.solve(r, phi=po, E=Eo), args.steps, args.warmup) / args.steps
        clk = clocks.stop()
        fd_bytes = 16 * prob.points      # read phi, write three field components (FP32)
        line.update({"metric": "finite-difference E at 256^3 FP32 (GB/s of phi read + E written)",
                     "value": fd_bytes / (per_fd * 1e-3) / 1e9, "unit": "GB/s", "ms_per_step": per_fd,
                     "config": {"workload": "E = -grad phi by centred differences on a 256^3 HE potential "
                                            "(8 anisotropic Gaussians, seed 1); FP64 direct-sum VGF solves",
                                "l2": "phi 67 MB read + E 201 MB written per step, 268 MB > 129 MB L2, no flush"},
                     "roofline": {"bound": "hbm", "kernel": "k_fd_gradient", "achieved": fd_bytes / (per_fd * 1e-3) / 1e9,
                                  "peak": peak, "unit": "GB/s", "frac": fd_bytes / (per_fd * 1e-3) / 1e9 / peak,
                                  "peak_kind": peak_kind, "traffic": None, "algorithmic_bytes": fd_bytes},
                     "direct_f64_ms_per_solve": direct,
                     "gpu_launches": args.steps, "clocks": clk})
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-context", action="store_true", help="skip the torch.fft (cuFFT) context timing")
    ap.add_argument("--workload", choices=["vgf256", "beam64", "gauss2d4096", "train128", "fd_direct"], default="vgf256",
                    help="vgf256 is the headline; the others print their own line (1 GPU)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "vgf256":
        return run_other(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
