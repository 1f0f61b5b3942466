#!/usr/bin/env python
"""Benchmark of the EA-ADC(3) Davidson sigma build sigma = M X on one GB300.

Workload (synthetic, the paper's molecules are not available): closed-shell
EA-ADC(3), nocc=40, nvir=400, naux=1400, mixed precision (tensor-core DF
ladder with split BF16 operands), a block of 4 trial vectors per step.  Metric: sigma-build TFLOP/s
counting the algorithmic DF-ladder work 4 naux nocc nvir^3 per trial vector
(the dominant term; the ring and coupling terms are not counted).  Inputs are
larger than L2 (B^Q alone is > 2 GB).  Also reported: end-to-end through the C
ABI with host buffers, the roofline of the tensor-core kernel timed live with
CUDA events, SM clocks sampled during the timed region, the CPU oracle on a
bounded sample, and the time to 4 roots with the Davidson solver.

--impl reference times the CPU oracle (the reference arm of this tier).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(nocc=40, nvir=400, naux=1400, order=3, kind="ea", nvec=4, nroots=4)
METRIC = "EA-ADC(3) sigma-build TFLOP/s (DF ladder 4*naux*nocc*nvir^3 per trial vector)"


def ladder_flops(o, v, naux, nvec):
    return 4.0 * naux * o * v ** 3 * nvec


def max_over_ranks(x, world, device=None):
    """The maximum of a per-rank float over all ranks (replicas: the slowest rank
    sets the step time); identity for one rank."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_tflops(flops_per_rank, ms, world):
    """Aggregate throughput of `world` replicas that each did flops_per_rank in ms."""
    return world * flops_per_rank / (ms / 1e3) / 1e12


def peaks():
    """(BF16 dense TF/s sustained, burst, HBM GB/s, source).  The ladder kernel is
    timed inside a seconds-long run of sigma steps (clocks settle under the power
    cap), so its roofline uses the sustained BF16 figure."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        burst = d.get("bf16_tflops", 1900.0)
        return d.get("bf16_tflops_sustained", burst), burst, d.get("hbm_gbs", 6800.0), "measured"
    return 1700.0, 1900.0, 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.gpu = gpu_index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for n, x in zip(names, r[5:9]):
                if x.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(sample_seconds=12.0):
    """The oracle's DF ladder (numpy) on a bounded sample of the same workload."""
    from adc_inputs import make_system
    from oracle.spinadapted import df_ladder

    w = WORKLOAD
    o, v, naux = w["nocc"], w["nvir"], w["naux"]
    rng = np.random.default_rng(0)
    # B^Q_vv of the same distribution (the ladder reads only this block)
    s = 0.3 / np.sqrt(naux)
    Bvv = np.empty((naux, v, v))
    for q in range(naux):
        g = rng.standard_normal((v, v))
        Bvv[q] = 0.5 * s * (g + g.T)
    X = rng.standard_normal((1, v, v))
    t0 = time.perf_counter()
    df_ladder(Bvv, X)
    t1 = time.perf_counter() - t0
    nmat = max(1, int(sample_seconds / max(t1, 1e-3)))
    X = rng.standard_normal((nmat, v, v))
    t0 = time.perf_counter()
    for k in range(nmat):
        df_ladder(Bvv, X[k:k + 1])
    dt = time.perf_counter() - t0
    flops = 4.0 * naux * v ** 3 * nmat
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"value": flops / dt / 1e12, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
            "sample": f"oracle DF ladder sum_Q B^Q Y_i B^Q for {nmat} of the {w['nvec'] * o} (vector, i) matrices "
                      f"(nvir={v}, naux={naux}); {dt:.1f} s", "seconds": dt}


def time_to_roots_medium(dev):
    """Setup + Davidson to 4 roots, FP64 plain vs mixed, EA-ADC(3) nocc=20 nvir=180 naux=600.

    Both runs converge to |dE| <= 1e-6 Eh between iterations and S-norm
    residual <= 1e-4; the mixed run is reported with the final refinement of
    its converged roots (other contractions FP32-accurate: refine=1, the
    default; FP64: refine=2) and without it, each root's |dE| against the
    FP64 run."""
    import torch

    from adc_inputs import make_system
    from paper_2012_06714_gb300 import ADC

    s = make_system(20, 180, 600, seed=0)
    out = {"workload": "EA- and IP-ADC(3) nocc=20 nvir=180 naux=600, 4 roots, tol 1e-6 Eh, residual 1e-4"}
    out["ip"] = time_to_roots_ip(dev, s)
    res = {}
    for name, prec, refine in (("fp64", "fp64", 0), ("mixed", "bf16x3", 1), ("mixed_refine_fp64", "bf16x3", 2),
                               ("mixed_unrefined", "bf16x3", 0)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g = ADC(torch.from_numpy(s.eps).to(dev), torch.from_numpy(s.B).to(dev), 20, order=3, kind="ea",
                precision=prec, res_tol=1e-4, refine=refine)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        e, p, _, st = g.davidson(4, tol=1e-6)
        t2 = time.perf_counter()
        g.close()
        res[name] = (e, p)
        out[name] = {"precision": prec, "setup_seconds": t1 - t0, "davidson_seconds": t2 - t1,
                     "total_seconds": t2 - t0, "iterations": st["iterations"], "sigma_vectors": st["sigma_vectors"],
                     "status": st["status"], "max_residual": st["max_residual"],
                     "refine_shift_eh": st["refine_shift"], "refine_seconds": st["refine_seconds"],
                     "energies_eh": [float(x) for x in e]}
    for name in ("mixed", "mixed_refine_fp64", "mixed_unrefined"):
        out[name]["abs_dE_eh_vs_fp64"] = [float(x) for x in np.abs(res["fp64"][0] - res[name][0])]
        out[name]["max_abs_dP_vs_fp64"] = float(np.abs(res["fp64"][1] - res[name][1]).max())
        out[name]["speedup_vs_fp64"] = out["fp64"]["total_seconds"] / out[name]["total_seconds"]
    return out


def time_to_roots_ip(dev, s):
    """IP-ADC(3) at nocc=20 nvir=180 naux=600, 4 roots: FP64 plain vs mixed precision (setup +
    Davidson; the mixed run continues with the accurate operator to residual 1e-6), each root's
    |dE| and |dP| against the FP64 run, and the IP sigma throughput of both (4 vectors)."""
    import torch

    from paper_2012_06714_gb300 import ADC

    o, v, naux = 20, 180, 600
    res, out = {}, {}
    for name, prec, kw in (("fp64", "fp64", dict(res_tol=1e-6)),
                           ("mixed", "bf16x3", dict(res_tol=1e-4, refine_res_tol=1e-6))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g = ADC(torch.from_numpy(s.eps).to(dev), torch.from_numpy(s.B).to(dev), o, order=3, kind="ip", precision=prec,
                **kw)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        e, p, _, st = g.davidson(4, tol=1e-8)
        t2 = time.perf_counter()
        X = torch.randn((4, g.dim), device=dev, dtype=torch.float64)
        S = torch.empty_like(X)
        g.sigma(X, out=S)
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        for _ in range(5):
            g.sigma(X, out=S)
        torch.cuda.synchronize()
        sig_ms = (time.perf_counter() - t3) / 5 * 1e3
        g.close()
        res[name] = (e, p)
        out[name] = {"setup_s": t1 - t0, "davidson_s": t2 - t1, "total_s": t2 - t0, "iterations": st["iterations"],
                     "sigma_vectors": st["sigma_vectors"], "status": st["status"], "max_residual": st["max_residual"],
                     "sigma_ms_4_vectors": sig_ms, "energies_eh": [float(x) for x in e]}
    out["mixed"]["abs_dE_eh_vs_fp64"] = [float(x) for x in np.abs(res["fp64"][0] - res["mixed"][0])]
    out["mixed"]["max_abs_dP_vs_fp64"] = float(np.abs(res["fp64"][1] - res["mixed"][1]).max())
    out["mixed"]["speedup_vs_fp64"] = out["fp64"]["total_s"] / out["mixed"]["total_s"]
    return out


def kernel_source_hash():
    """sha256 of the device code of the ladder kernel (csrc/ladder_tc.cu up to its host part)."""
    import hashlib

    src = open(os.path.join(ROOT, "paper_2012_06714_gb300", "csrc", "ladder_tc.cu")).read()
    return hashlib.sha256(src.split("// ---- host: tensor maps")[0].encode()).hexdigest()


def profiled_traffic():
    """DRAM bytes per DF-ladder GEMM launch from the committed ncu summary, or None
    when the kernel's device code has changed since the counters were taken."""
    p = os.path.join(ROOT, "profiles", "k_gemm_ladder_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    return d.get("dram_bytes_per_launch") if d.get("device_code_sha256") == kernel_source_hash() else None


def fp64_plain_profile():
    """The FP64-plain comparator at this workload, measured by `bench.py --fp64-plain` (its FP64 setup
    alone takes minutes on GB300's FP64 units, so it is not rerun here) and committed under
    profiles/; None if absent."""
    p = os.path.join(ROOT, "profiles", "fp64_plain_ea3_o40_v400_Q1400.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    f = d.get("fp64", {})
    return {"source": "profiles/fp64_plain_ea3_o40_v400_Q1400.json (bench.py --fp64-plain)",
            "setup_s": f.get("setup_s"), "sigma_s_per_vector": f.get("sigma_s_per_vector"),
            "time_to_roots_s_extrapolated": f.get("time_to_roots_s_extrapolated"),
            "mixed_total_s_same_run": d.get("mixed", {}).get("total_s"),
            "speedup_mixed_vs_fp64_same_run": d.get("speedup_mixed_vs_fp64")}


def large_workload_profile():
    """The 1028-MO workload (EA-ADC(3), nocc=68, nvir=960, naux=3000), measured by `bench.py --large`
    and committed under profiles/ (setup and solve take about eleven minutes and 254 GB, so it is
    not rerun by the default bench); None if absent."""
    p = os.path.join(ROOT, "profiles", "large_ea3_o68_v960_Q3000.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    sg, tr = d.get("sigma", {}), d.get("time_to_roots", {})
    return {"source": "profiles/large_ea3_o68_v960_Q3000.json (bench.py --large)", "workload": d.get("case"),
            "setup_s": d.get("setup_s"), "sigma_ms_per_step": sg.get("ms_per_step"), "sigma_tflops": sg.get("tflops"),
            "ladder_tflops": sg.get("ladder_tflops"),
            "ladder_frac_of_sustained_bf16_over_3": sg.get("ladder_frac_of_sustained_bf16_over_3"),
            "time_to_4_roots_s": tr.get("seconds"), "sigma_vectors": tr.get("sigma_vectors"),
            "status": tr.get("status"), "s_symmetry_rel": d.get("s_symmetry_rel"),
            "peak_memory_mib": (d.get("memory") or {}).get("peak_used_mib")}


def run_ladder_case(args):
    """Small profiling case of the ladder kernel (for ncu): EA-ADC(3) with
    nocc=4, nvir=400, naux=400 and 40 trial vectors, i.e. 160 ladder matrices
    per sigma call -- the same per-launch GEMM shapes as the bench workload
    (160 matrices, 40 auxiliary functions per chunk) with a few GB on the
    device.  Runs `--steps` sigma calls after one warm-up call and prints the
    ladder launch timing of the last call."""
    import torch

    from adc_inputs import make_system
    from paper_2012_06714_gb300 import ADC

    o, v, naux, nvec = 4, 400, 400, 40
    s = make_system(o, v, naux, seed=0)
    # contractions=1: the non-ladder terms off the tensor-core kernel, so that every k_gemm_pair
    # launch is a ladder GEMM (setup: 2 ladders x 2 launches; each sigma: 10 chunks x 2)
    g = ADC(torch.from_numpy(s.eps).cuda(), torch.from_numpy(s.B).cuda(), o, order=3, kind="ea",
            precision="bf16x3", contractions=1)
    X = torch.randn(nvec, g.dim, device="cuda", dtype=torch.float64)
    S = torch.empty_like(X)
    g.sigma(X, out=S)
    for _ in range(max(1, args.steps) - 1):
        g.sigma(X, out=S)
    torch.cuda.synchronize()
    g.kernel_timing(True)
    g.sigma(X, out=S)
    kt = g.kernel_timing(False)
    print(json.dumps({"case": "ladder o=4 v=400 naux=400 nvec=40", "launches": kt["launches"], "ms": kt["ms"],
                      "algo_tflops": kt["algo_flops"] / kt["ms"] / 1e9,
                      "mma_tflops": kt["mma_flops"] / kt["ms"] / 1e9}))
    g.close()
    return 0


def run_ladder_large(args):
    """The DF-ladder kernel at the per-launch shapes of the largest workload, EA-ADC(3) with
    nocc=68, nvir=960, naux=3000 (1028 MOs), 4 trial vectors: 4 x 68 = 272 ladder matrices of
    960 x 960 per sigma step.  That workload's setup does not fit one GPU as the handle is laid
    out (its o^2 v^2 tensors are 34 GB each), so the ladder runs in a handle with nocc=4 and
    68 trial vectors -- the same 272 matrices and the same B^Q (960 x 960 x 3000), hence the same
    GEMM launches and flops (4 naux nvir^3 per matrix).  Reports the ladder GEMMs' live
    CUDA-event throughput over `--steps` sigma calls after one warm-up call."""
    import torch

    from adc_inputs import make_system
    from paper_2012_06714_gb300 import ADC

    torch.cuda.set_device(0)
    o, v, naux, nvec = 4, 960, 3000, 68
    s = make_system(o, v, naux, seed=0)
    t0 = time.perf_counter()
    g = ADC(torch.from_numpy(s.eps).cuda(), torch.from_numpy(s.B).cuda(), o, order=3, kind="ea", precision="bf16x3",
            tune_cache=args.tune_cache)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    X = torch.randn((nvec, g.dim), device="cuda", dtype=torch.float64) / np.sqrt(g.dim)
    S = torch.empty_like(X)
    g.sigma(X, out=S)
    torch.cuda.synchronize()
    g.kernel_timing(True)
    t0 = time.perf_counter()
    for _ in range(max(1, args.steps)):
        g.sigma(X, out=S)
    torch.cuda.synchronize()
    wall = (time.perf_counter() - t0) / max(1, args.steps)
    kt = g.kernel_timing(False)
    g.close()
    steps = max(1, args.steps)
    bf16_peak, bf16_burst, _, src = peaks()
    lt = kt["ladder_algo_flops"] / (kt["ladder_ms"] / 1e3) / 1e12
    out = {"case": "DF ladder at the 1028-MO shapes: nvir=960, naux=3000, 272 matrices per sigma "
                   "(4 vectors x 68 occupied of EA-ADC(3) 68/960/3000), run as nocc=4 x 68 vectors",
           "ladder_flops_per_sigma": kt["ladder_algo_flops"] / steps, "ladder_ms_per_sigma": kt["ladder_ms"] / steps,
           "ladder_launches_per_sigma": kt["ladder_launches"] / steps, "ladder_tflops": lt,
           "frac_of_sustained_bf16_over_3": lt / (bf16_peak / 3.0), "peak_source": src,
           "sigma_wall_s": wall, "setup_s": setup_s}
    print(json.dumps(out))
    return 0


class MemorySampler:
    """Peak device memory in use (nvidia-smi, every 200 ms) while a phase runs."""

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.gpu = gpu_index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", "--query-gpu=memory.used,memory.total",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        used, total = [], []
        for r in self.f.read().strip().splitlines():
            try:
                a, b = (float(x) for x in r.split(","))
            except ValueError:
                continue
            used.append(a)
            total.append(b)
        if not used:
            return None
        return {"peak_used_mib": max(used), "total_mib": max(total), "samples": len(used)}


def run_large(args):
    """The 1028-MO workload end to end: EA-ADC(3), nocc=68, nvir=960, naux=3000 (B^Q 25 GB in
    FP64), mixed precision in the lean layout (the o^2 v^2 tensors are 34 GB each in FP64),
    4 roots with a subspace of up to 16 vectors per root.  Reports setup time, the sigma step
    of 4 trial vectors (ladder TFLOP/s timed live with CUDA events), the S-symmetry of M at
    this size (x0^T S M x1 = x1^T S M x0, a parity property that holds at any size), the time
    to 4 roots and the peak device memory."""
    import torch

    from adc_inputs import make_system
    from paper_2012_06714_gb300 import ADC

    torch.cuda.set_device(0)
    o, v, naux, nvec = 68, 960, 3000, 4
    need = 8.0 * naux * (o + v) ** 2  # the host copy of B^Q
    try:
        avail = float([ln.split()[1] for ln in open("/proc/meminfo") if ln.startswith("MemAvailable")][0]) * 1024
    except (OSError, IndexError, ValueError):
        avail = 0.0
    if avail < 2.0 * need:
        print(json.dumps({"case": "1028-MO workload", "unavailable": f"host memory {avail / 1e9:.0f} GB available, "
                                                                     f"{2 * need / 1e9:.0f} GB wanted"}))
        return 1
    t0 = time.perf_counter()
    s = make_system(o, v, naux, seed=0)
    gen_s = time.perf_counter() - t0
    mem = MemorySampler(torch.cuda.current_device())
    mem.start()
    t0 = time.perf_counter()
    g = ADC(s.eps, s.B, o, order=3, kind="ea", precision="bf16x3", lean=1, res_tol=1e-4, max_space_per_root=16,
            keep_per_root=4, nguess_extra=0, max_iter=200, tune_cache=args.tune_cache)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    del s
    mp = g.mp_energy()
    phases = g.get("setup_seconds", (8,))
    out = {"case": "EA-ADC(3) nocc=68 nvir=960 naux=3000 (1028 MOs), bf16x3, lean layout", "setup_s": setup_s,
           "setup_phases_s": dict(zip(["inputs_and_ladder_planes", "integrals", "amplitudes_E2", "ladder_of_t",
                                       "t2_2_rest_t1_2_E3", "one_particle_block", "transition_parts_diag", "total"],
                                      (float(x) for x in phases))),
           "input_generation_s": gen_s, "dim": g.dim, "mp_energy_eh": list(mp)}
    gen = torch.Generator(device="cuda").manual_seed(1)
    X = torch.randn((nvec, g.dim), device="cuda", dtype=torch.float64, generator=gen) / np.sqrt(g.dim)
    S = torch.empty_like(X)
    g.sigma(X, out=S)
    torch.cuda.synchronize()
    # S-symmetry: (S x)_1p = x_1p, (S x)_2p1h = 2 Y - Y(ab swap)

    def apply_S(x):
        y2 = x[v:].view(o, v, v)
        return torch.cat([x[:v], (2.0 * y2 - y2.transpose(1, 2)).reshape(-1)])

    a = float(X[0] @ apply_S(S[1]))
    b = float(X[1] @ apply_S(S[0]))
    scale = float(np.sqrt(abs(float(X[0] @ apply_S(S[0]))) * abs(float(X[1] @ apply_S(S[1])))))
    out["s_symmetry_rel"] = abs(a - b) / scale
    out["sigma_finite"] = bool(torch.isfinite(S).all())
    g.kernel_timing(True)
    steps = max(1, args.steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        g.sigma(X, out=S)
    e1.record()
    torch.cuda.synchronize()
    kt = g.kernel_timing(False)
    ms = e0.elapsed_time(e1) / steps
    # the other tensor-core contractions by shape (milliseconds summed over launches; K slices
    # of one contraction run concurrently on side streams, so their sum exceeds their wall time)
    shapes = {}
    for M, N, K, BN, fl, lms, lad in g.kernel_launches():
        if not lad:
            a = shapes.setdefault(f"M{int(M)} N{int(N)} K{int(K)}", [0, 0.0, 0.0])
            a[0] += 1
            a[1] += fl / steps
            a[2] += lms / steps
    top = sorted(shapes.items(), key=lambda kv: -kv[1][2])[:12]
    bf16_peak, bf16_burst, _, src = peaks()
    lt = kt["ladder_algo_flops"] / (kt["ladder_ms"] / 1e3) / 1e12
    out["sigma"] = {"ms_per_step": ms, "tflops": ladder_flops(o, v, naux, nvec) / (ms / 1e3) / 1e12,
                    "ladder_tflops": lt, "ladder_frac_of_sustained_bf16_over_3": lt / (bf16_peak / 3.0),
                    "ladder_ms_per_step": kt["ladder_ms"] / steps, "peak_source": src,
                    "other_tensor_core_ms_per_step": (kt["ms"] - kt["ladder_ms"]) / steps,
                    "other_tensor_core_tflops": (kt["algo_flops"] - kt["ladder_algo_flops"])
                    / max(kt["ms"] - kt["ladder_ms"], 1e-9) / 1e9,
                    "launches_per_step": kt["kernels"] / steps,
                    "other_by_shape": {k: {"launches": n // steps, "ms": t, "tflops": fl / max(t, 1e-9) / 1e9}
                                       for k, (n, fl, t) in top}}
    del X, S
    torch.cuda.empty_cache()
    t0 = time.perf_counter()
    e, p, _, st = g.davidson(4, tol=1e-6)
    out["time_to_roots"] = {"seconds": time.perf_counter() - t0, "setup_seconds": setup_s,
                            "subspace": "<= 16 vectors per root, restart onto 4 per root; |dE| <= 1e-6 Eh, "
                                        "residual 1e-4, then one accurate-operator Rayleigh-Ritz step",
                            "energies_eh": [float(x) for x in e], "spectroscopic_factors": [float(x) for x in p],
                            "iterations": st["iterations"], "sigma_vectors": st["sigma_vectors"],
                            "sigma_seconds": st["sigma_seconds"], "max_residual": st["max_residual"],
                            "status": st["status"], "refine_shift_eh": st["refine_shift"],
                            "refine_seconds": st["refine_seconds"]}
    out["memory"] = mem.stop()
    g.close()
    print(json.dumps(out))
    return 0


def run_davidson_case(args):
    """Small profiling case of the Davidson subspace kernels (for ncu):
    EA-ADC(3) mixed precision with nocc=24, nvir=240, naux=500 (1.38e6-element
    vectors, so a subspace of 16-32 vectors exceeds L2; about 2.5 GB on the
    device), 4 roots, at most 8 vectors per root, `--steps` Davidson
    iterations (not converged; the status is printed)."""
    import torch

    from adc_inputs import make_system
    from paper_2012_06714_gb300 import ADC

    o, v, naux = 24, 240, 500
    s = make_system(o, v, naux, seed=0)
    g = ADC(torch.from_numpy(s.eps).cuda(), torch.from_numpy(s.B).cuda(), o, order=3, kind="ea",
            precision="bf16x3", max_iter=max(1, args.steps), refine=0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e, p, _, st = g.davidson(4, tol=1e-12)
    print(json.dumps({"case": "davidson EA-ADC(3) o=24 v=240 naux=500, 4 roots", "dim": g.dim,
                      "iterations": st["iterations"], "sigma_vectors": st["sigma_vectors"],
                      "seconds": time.perf_counter() - t0, "sigma_seconds": st["sigma_seconds"],
                      "status": st["status"]}))
    g.close()
    return 0


def run_fp64_plain(args):
    """The plain FP64 comparator at the bench workload (EA-ADC(3), nocc=40 nvir=400 naux=1400,
    4 roots): the mixed-precision solve to 4 roots is run and timed in full (setup + Davidson +
    refinement + spectroscopic factors); the FP64 path's setup is timed in full and its sigma
    on a bounded sample (2 calls of 2 vectors), and its time to 4 roots is extrapolated as
    setup + (sigma vectors of the mixed solve) x (FP64 seconds per sigma vector) + the mixed
    solve's non-sigma Davidson time (the same FP64 subspace work on both paths)."""
    import torch

    from adc_inputs import make_system
    from paper_2012_06714_gb300 import ADC

    torch.cuda.set_device(0)
    w = WORKLOAD
    o, v, naux = w["nocc"], w["nvir"], w["naux"]
    s = make_system(o, v, naux, seed=0)
    out = {"workload": f"EA-ADC(3) nocc={o} nvir={v} naux={naux}, 4 roots, |dE| <= 1e-6 Eh, residual 1e-4"}
    eps, B = torch.from_numpy(s.eps).cuda(), torch.from_numpy(s.B).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = ADC(eps, B, o, order=3, kind="ea", precision="bf16x3", res_tol=1e-4, max_space_per_root=16, keep_per_root=4)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    e, p, _, st = g.davidson(4, tol=1e-6)
    t2 = time.perf_counter()
    g.close()
    mixed = {"setup_s": t1 - t0, "davidson_s": t2 - t1, "total_s": t2 - t0, "sigma_vectors": st["sigma_vectors"],
             "sigma_s": st["sigma_seconds"], "iterations": st["iterations"], "energies_eh": [float(x) for x in e],
             "spectroscopic_factors": [float(x) for x in p]}
    out["mixed"] = mixed
    t0 = time.perf_counter()
    g = ADC(eps, B, o, order=3, kind="ea", precision="fp64", res_tol=1e-4)
    torch.cuda.synchronize()
    setup64 = time.perf_counter() - t0
    X = torch.randn((2, g.dim), device="cuda", dtype=torch.float64) / np.sqrt(g.dim)
    S = torch.empty_like(X)
    g.sigma(X, out=S)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.sigma(X, out=S)
    torch.cuda.synchronize()
    per_vec = (time.perf_counter() - t0) / 2
    g.close()
    other = mixed["davidson_s"] - mixed["sigma_s"]
    est = setup64 + mixed["sigma_vectors"] * per_vec + other
    out["fp64"] = {"setup_s": setup64, "sigma_s_per_vector": per_vec,
                   "sigma_tflops": 4.0 * naux * o * v ** 3 / per_vec / 1e12,
                   "time_to_roots_s_extrapolated": est,
                   "note": "setup measured; sigma measured on 2 calls of 2 vectors; time to roots = setup + "
                           "mixed sigma-vector count x FP64 sigma seconds per vector + the mixed run's non-sigma "
                           "Davidson seconds"}
    out["speedup_mixed_vs_fp64"] = est / mixed["total_s"]
    print(json.dumps(out))
    return 0


def run_batched(args):
    """The batched IP-ADC(3) workload: 64 synthetic molecules (nocc ~ U{8..30}, nvir ~ U{60..250},
    naux = 3.5 nmo, seeds 0..63), mixed precision, 6 roots each, set up and solved as one batch
    (adc_setup_batch / adc_davidson_batch: each system on its own stream and host thread) and one
    at a time on the same GPU; wall times of both, and the largest root difference between them."""
    import torch

    from adc_inputs import batched_ip_molecules, make_system
    from paper_2012_06714_gb300 import ADC, ADCBatch

    torch.cuda.set_device(0)
    mols = batched_ip_molecules(args.nmol)
    systems = []
    for m in mols:
        s = make_system(m["nocc"], m["nvir"], m["naux"], seed=m["seed"])
        systems.append((s.eps, s.B, m["nocc"]))
    # the workload's mixed precision with FP32-accurate setup contractions (contractions=2; the
    # FP64 setup that IP handles take by default costs o^3 v^3 FP64 flop per molecule)
    opts = dict(res_tol=1e-4, max_iter=300, max_space_per_root=24, keep_per_root=4, contractions=2)
    # library first use (handles, module loading) outside the timed regions
    ADC(systems[0][0], systems[0][1], systems[0][2], order=3, kind="ip", precision="bf16x3").close()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b = ADCBatch(systems, order=3, kind="ip", precision="bf16x3", **opts)
    t1 = time.perf_counter()
    e, p, st, status = b.davidson(6, tol=1e-6)
    t2 = time.perf_counter()
    b.close()
    # the same batch with each handle's sigma captured as CUDA graphs
    torch.cuda.synchronize()
    g0 = time.perf_counter()
    b = ADCBatch(systems, order=3, kind="ip", precision="bf16x3", cuda_graphs=1, **opts)
    g1 = time.perf_counter()
    eg, _, stg, statusg = b.davidson(6, tol=1e-6)
    g2 = time.perf_counter()
    b.close()
    seq_setup = seq_solve = 0.0
    dmax = 0.0
    for k, (eps, B, o) in enumerate(systems):
        t3 = time.perf_counter()
        g = ADC(eps, B, o, order=3, kind="ip", precision="bf16x3", **opts)
        t4 = time.perf_counter()
        e1, _, _, _ = g.davidson(6, tol=1e-6)
        t5 = time.perf_counter()
        g.close()
        seq_setup += t4 - t3
        seq_solve += t5 - t4
        dmax = max(dmax, float(np.abs(e[k] - e1).max()))
    out = {"workload": f"batched IP-ADC(3), {len(systems)} molecules, nocc 8..30, nvir 60..250, naux 3.5 nmo, "
                       "6 roots, bf16x3 (setup FP32-accurate), |dE| <= 1e-6 Eh, residual 1e-4",
           "batched": {"setup_s": t1 - t0, "solve_s": t2 - t1, "total_s": t2 - t0,
                       "converged": int((status == 0).sum()), "sigma_vectors": int(st[:, 1].sum())},
           "batched_cuda_graphs": {"setup_s": g1 - g0, "solve_s": g2 - g1, "total_s": g2 - g0,
                                   "converged": int((statusg == 0).sum()),
                                   "max_abs_dE_vs_batched_eh": float(np.abs(eg - e).max())},
           "one_at_a_time": {"setup_s": seq_setup, "solve_s": seq_solve, "total_s": seq_setup + seq_solve},
           "max_abs_dE_batched_vs_one_at_a_time_eh": dmax}
    out["speedup"] = out["one_at_a_time"]["total_s"] / out["batched"]["total_s"]
    print(json.dumps(out))
    return 0


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = WORKLOAD
    vals = []
    for _ in range(args.warmup):
        cpu_baseline(sample_seconds=2.0)
    for _ in range(args.steps):
        vals.append(cpu_baseline(sample_seconds=8.0))
    v = float(np.mean([x["value"] for x in vals]))
    cb = dict(vals[-1])
    cb["value"] = v
    ms = float(np.mean([x["seconds"] for x in vals])) * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "EA-ADC(3) nocc=40 nvir=400 naux=1400, CPU oracle DF ladder sample",
                       **{k: w[k] for k in ("nocc", "nvir", "naux", "order", "kind", "nvec")}},
            "cpu_baseline": cb, "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist

    from adc_inputs import make_system
    from paper_2012_06714_gb300 import ADC

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    def barrier():
        if world > 1:
            dist.barrier()

    w = WORKLOAD
    o, v, naux, nvec = w["nocc"], w["nvir"], w["naux"], w["nvec"]
    sysm = make_system(o, v, naux, seed=0)
    eps_d = torch.from_numpy(sysm.eps).to(dev)
    B_d = torch.from_numpy(sysm.B).to(dev)
    # first use of the library in this process (CUDA/cuBLAS handles, module loading), timed apart
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tiny = make_system(2, 8, 16, seed=0)
    ADC(torch.from_numpy(tiny.eps).to(dev), torch.from_numpy(tiny.B).to(dev), 2, order=3, kind="ea",
        precision="bf16x3").close()
    torch.cuda.synchronize()
    cold_start_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    # tile autotuner: a fresh cache unless one is given, so the tiles are measured in the first warm-up step
    tune_cache = args.tune_cache or os.path.join(tempfile.mkdtemp(prefix="adc_tiles_"), "tiles.txt")
    gpu = ADC(eps_d, B_d, o, order=3, kind="ea", precision="bf16x3", res_tol=1e-4, tune_cache=tune_cache)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    del B_d
    stream = torch.cuda.current_stream()
    gpu.set_stream(stream.cuda_stream)
    gen = torch.Generator(device=dev).manual_seed(1 + rank)
    X = torch.randn((nvec, gpu.dim), device=dev, dtype=torch.float64, generator=gen) / np.sqrt(gpu.dim)
    S = torch.empty_like(X)
    for _ in range(max(3, args.warmup)):
        gpu.sigma(X, out=S)
    torch.cuda.synchronize()

    clocks = Clocks(torch.cuda.current_device())
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        gpu.sigma(X, out=S)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1) / args.steps
    clk = clocks.stop()
    ms = max_over_ranks(ms, world, dev)
    flops = ladder_flops(o, v, naux, nvec)
    value = whole_job_tflops(flops, ms, world)

    # roofline of the tensor-core ladder kernel, timed live with CUDA events
    gpu.kernel_timing(True)
    nprof = 2
    for _ in range(nprof):
        gpu.sigma(X, out=S)
    kt = gpu.kernel_timing(False)
    launches_per_step = kt["kernels"] / nprof
    bf16_peak, bf16_burst, hbm_peak, peak_src = peaks()
    peak = bf16_peak / 3.0  # three BF16 products per split-precision product
    # the dominant kernel: k_gemm_pair in its DF-ladder role (both GEMMs of the ladder)
    achieved = kt["ladder_algo_flops"] / (kt["ladder_ms"] / 1e3) / 1e12
    traffic = profiled_traffic()
    roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": traffic, "kernel": "k_gemm_pair, DF-ladder GEMMs (GEMM1 + GEMM2, cta_group::2)",
            "peak_note": f"{peak_src} sustained BF16 dense {bf16_peak:.1f} TF/s / 3 split products "
                         f"(burst {bf16_burst:.1f} TF/s: frac {achieved / (bf16_burst / 3.0):.3f})",
            "tensor_pipe_frac": kt["ladder_mma_flops"] / (kt["ladder_ms"] / 1e3) / 1e12 / bf16_peak,
            "launches_per_step": kt["ladder_launches"] / nprof,
            "ms_per_launch": kt["ladder_ms"] / max(kt["ladder_launches"], 1),
            "other_tensor_core_contractions": {
                "launches_per_step": (kt["launches"] - kt["ladder_launches"]) / nprof,
                "ms_per_step": (kt["ms"] - kt["ladder_ms"]) / nprof,
                "algo_tflops": (kt["algo_flops"] - kt["ladder_algo_flops"]) / max(kt["ms"] - kt["ladder_ms"], 1e-9) / 1e9}}
    # end to end through the C ABI with pinned host buffers (copies inside the timed region)
    Xh = torch.empty((nvec, gpu.dim), dtype=torch.float64, pin_memory=True)
    Xh.copy_(X.cpu())
    Sh = torch.empty_like(Xh).pin_memory()
    lib = gpu._lib
    import ctypes

    def sig_host():
        rc = lib.adc_sigma(gpu._h, ctypes.c_void_p(Xh.data_ptr()), ctypes.c_void_p(Sh.data_ptr()), nvec, 0)
        assert rc == 0

    sig_host()
    ke = max(2, args.steps // 2)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(ke):
        sig_host()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / ke, world, dev)
    e2e = {"value": world * flops / e2e_s / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": int(Xh.numel() * 8),
           "d2h_bytes_per_step": int(Sh.numel() * 8)}

    # time to 4 roots (Davidson): mixed precision at this workload, and FP64 plain vs mixed on the
    # nocc=20 nvir=180 naux=600 workload where the FP64 path is affordable on GB300's FP64 units
    roots = None
    if not args.no_roots:
        # subspace of up to 16 vectors per root, thick restart onto 4 per root
        gpu.set_options(max_space_per_root=16, keep_per_root=4)
        t0 = time.perf_counter()
        e, p, _, st = gpu.davidson(w["nroots"], tol=1e-6)
        roots = {"workload": "nocc=40 nvir=400 naux=1400, bf16x3", "seconds": time.perf_counter() - t0,
                 "subspace": "<= 16 vectors per root, restart onto 4 per root; |dE| <= 1e-6 Eh, residual 1e-4",
                 "setup_seconds": setup_s, "library_first_use_seconds": cold_start_s,
                 "energies_eh": [float(x) for x in e],
                 "spectroscopic_factors": [float(x) for x in p], "iterations": st["iterations"],
                 "sigma_vectors": st["sigma_vectors"], "sigma_seconds": st["sigma_seconds"],
                 "max_residual": st["max_residual"], "status": st["status"],
                 "refine_shift_eh": st["refine_shift"], "refine_seconds": st["refine_seconds"]}
        roots["fp64_vs_mixed"] = time_to_roots_medium(dev)
        roots["fp64_plain_this_workload"] = fp64_plain_profile()

    line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16x3", "data": "synthetic",
            "config": {"workload": "EA-ADC(3) sigma build, nocc=40 nvir=400 naux=1400, 4 trial vectors",
                       "nocc": o, "nvir": v, "naux": naux, "order": 3, "kind": "ea", "nvec": nvec, "dim": gpu.dim,
                       "l2": "inputs larger than L2 (B^Q > 2 GB)", "parallelism": "replicas" if world > 1 else "1 GPU",
                       "tiles": "autotuned in the first warm-up step (adc_options.tune_cache)"},
            "e2e": e2e, "roofline": roof, "gpu_launches": int(round(launches_per_step)), "clocks": clk,
            "time_to_roots": roots, "large_workload": large_workload_profile()}
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line))
    gpu.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-roots", action="store_true")
    ap.add_argument("--ladder-case", action="store_true", help="small ladder profiling case (for ncu)")
    ap.add_argument("--davidson-case", action="store_true", help="small Davidson profiling case (for ncu)")
    ap.add_argument("--batched", action="store_true", help="batched IP-ADC(3) workload (64 molecules)")
    ap.add_argument("--ladder-large", action="store_true",
                    help="ladder kernel at the per-launch shapes of the 1028-MO workload")
    ap.add_argument("--large", action="store_true",
                    help="the 1028-MO workload end to end (setup, sigma, time to 4 roots) in the lean layout")
    ap.add_argument("--nmol", type=int, default=64)
    ap.add_argument("--tune-cache", default=None,
                    help="tile autotuner cache file (tiles measured in the first warm-up step)")
    ap.add_argument("--fp64-plain", action="store_true",
                    help="FP64 comparator at the bench workload (setup timed, time to roots extrapolated)")
    args = ap.parse_args()
    if args.davidson_case:
        return run_davidson_case(args)
    if args.fp64_plain:
        return run_fp64_plain(args)
    if args.batched:
        return run_batched(args)
    if args.ladder_large:
        return run_ladder_large(args)
    if args.large:
        return run_large(args)
    if args.ladder_case:
        return run_ladder_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
