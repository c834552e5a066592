#!/usr/bin/env python
"""Benchmark of the fused thermal D3Q19 lattice Boltzmann step on GB300.

Headline workload: the paper-geometry boiling cell 512^3 (L = 512 as in the paper's Table 1;
rho = 1.50 (1 + 0.01 xi) inside coexistence between a hot bottom and a cold top wall, Pr = 9,
Ra = half the largest value the adiabatic gradient allows at L = 512), FP32 form. The FP16- and
BF16-deviation and FP64 forms of the same cell are timed beside it and stated with their error
against the FP64 step. One "step" is one full time step of the method (pull streaming, moments,
psi, force, velocities, divergence, f and g collisions, walls) = one fused kernel launch.
Value = lattice-node updates per second (GLUPS) of the whole job.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

With N > 1 (torchrun) every rank runs an independent replica of the cell (the path has no
collective at one GPU per process); value = all ranks' node updates / max rank time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "GLUPS and % HBM roofline per full step; mixed vs FP64 at stated error"
UNIT = "GLUPS"
Q = 19
FORMS = {"f64": 0, "f32": 1, "bf16dev": 2, "fp16dev": 3, "fp16loc": 4}
STORE_BYTES = {"f64": 8, "f32": 4, "bf16dev": 2, "fp16dev": 2, "fp16loc": 2}
# values stored per lattice and node: the 19 populations, plus two reference slots for the FP16
# storage against local references (its extra traffic counts against its roofline fraction)
STORED_SLOTS = {"f64": 19, "f32": 19, "bf16dev": 19, "fp16dev": 19, "fp16loc": 21}
# forms whose traffic is the 76 values per node of the yardstick lb_stream_bound (the FP64 form is
# bound by its FP64 pipe; the local-reference form also loads the source nodes' references)
PATTERN_FORMS = ("f32", "fp16dev", "bf16dev")
KERNEL_TYPE = {"f64": "double", "f32": "float", "bf16dev": "__nv_bfloat16", "fp16dev": "__half",
               "fp16loc": "tlbm::half_loc"}

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the fused step
# kernel from an ncu capture of a smaller cell (`nodes` nodes; a capture with more than the
# launch time is kept to a few GB on the device), keyed by the hash of the kernel sources it
# was taken on. The headline's traffic is that capture scaled by the node count (the traffic
# of one launch grows in proportion to the nodes it updates); null once the sources changed.
TRAFFIC = {"src_hash": "89f84465a4989b8a", "nodes": 192 ** 3,
           "bytes_per_launch": {"f32": 1148334592 + 1032008960, "fp16loc": 602396672 + 553547520,
                                "fp16dev": 543652608 + 495205632},
           "what": "ncu DRAM bytes of one launch of the 192^3 paper-geometry cell, scaled by the node count"}

# FP64 operations per node of one FP64 step (ncu: 2 x DFMA + DADD + DMUL thread instructions of
# one step of the 128^3 single-phase cell, i.e. the per-node pre-pass lb_fields_kernel,
# 2 x 39,845,888 + 100,663,296, plus the step kernel, 2 x 327,282,688 + 91,111,424 + 129,517,568,
# divided by its 2,097,152 nodes; the step kernel's count includes its chunk prologues, a smaller
# share at 512^3), and GB300's nominal FP64 rate (152 SMs x 2 FP64 FMA per clock x 2 flops x 2.07
# GHz = 1.26 TFLOP/s; no measured FP64 peak).
FP64_FLOPS_PER_NODE = (2 * (39845888 + 327282688) + (100663296 + 91111424) + 129517568) / 2097152
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


STEP_KERNEL_SOURCES = ("lb_kernels.cuh", "lb_launch.cuh", "lb_prec_f32.cu", "lb_prec_f16.cu")


def kernel_src_hash() -> str:
    """Hash of the sources the step kernels are compiled from (the FP32 and FP16 forms)."""
    h = hashlib.sha256()
    for name in STEP_KERNEL_SOURCES:
        h.update((ROOT / "paper_1111_0905_gb300" / "csrc" / name).read_bytes())
    return h.hexdigest()[:16]


def measured_peaks() -> dict:
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return {"hbm_gbs": float(d["hbm_gbs"]), "src": "measured"}
    return {"hbm_gbs": 6800.0, "src": "fallback"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms while running."""

    Q = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        self.file = None

    def __enter__(self):
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        cmd = ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "100"]
        if self.uuid:
            cmd.insert(1, f"--id={self.uuid}")
        try:
            self.proc = subprocess.Popen(cmd, stdout=self.file, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except FileNotFoundError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        self.file.flush()

    def summary(self) -> dict:
        rows = []
        try:
            for line in Path(self.file.name).read_text().splitlines():
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 10:
                    rows.append(parts)
        finally:
            os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        smax = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[6 + k].lower() == "active"})
        busy = [s for s in sm if s > 0.5 * (max(smax) if smax else 1)] or sm
        return {"sm_mhz": statistics.median(busy) if busy else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


def replica_aggregate(local_ms: float, nodes_per_rank: int, steps: int, ws: int, device="cpu"):
    """Whole-job result of N independent replicas: the max over ranks of the timed milliseconds
    and the whole-job GLUPS = all ranks' node updates / that max time (weak scaling)."""
    import torch
    ms = local_ms
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([local_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, nodes_per_rank * steps * ws / (ms * 1e-3) / 1e9


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


HEADLINE_N = 512
# Forms timed at the headline size, the headline form first. FP64 is bound by its FP64
# instructions (about 134 ms per step at 512^3), so it is timed over fewer steps.
FORM_ORDER = ("f32", "fp16loc", "fp16dev", "bf16dev", "f64")
F64_MAX_STEPS = 20
ERR_STEPS_HEADLINE = 100
C5_STEPS = 1000


def workload(prec_name: str, n: int = HEADLINE_N):
    """The paper-geometry boiling cell (n^3; 512^3 is the headline), or with n = 128 the
    single-phase convection cell."""
    from paper_1111_0905_gb300 import config
    if n == 128:
        return config.single_phase_cell(128, precision=FORMS[prec_name])
    return config.paper_scale_cell(n, precision=FORMS[prec_name])


def describe(w) -> str:
    p = w.params
    if w.kind == "boiling":
        return (f"paper-geometry boiling cell {p.nx}x{p.ny}x{p.nz} (rho = 1.50 (1 + 0.01 xi) inside "
                f"coexistence, T_d/T_u = T_m (1 +- 0.05), tau_nu = {p.tau_nu:g}, tau_kappa = "
                f"{p.tau_kappa:g}, Pr = 9, Ra = 0.5 Ra_max(L = {p.nz}))")
    return (f"single-phase thermal convection cell {p.nx}x{p.ny}x{p.nz} (rho = 2.30, Pr = 9, "
            f"tau_nu = {p.tau_nu:g}, tau_kappa = {p.tau_kappa:g}, Ra = 0.5 Ra_max)")


def config_dict(w, form: str) -> dict:
    p = w.params
    N = p.nx * p.ny * p.nz
    in_bytes = 2 * Q * N * STORE_BYTES[form]
    return {"workload": f"{describe(w)}, {form} form",
            "grid": [p.nx, p.ny, p.nz], "nodes": N, "form": form,
            "l2": f"inputs larger than L2: {in_bytes / 1e9:.2f} GB of populations read per step "
                  f"> 129 MB L2; no flush",
            "parallelism": "replicas", "lattice": "D3Q19 x2 (f, g)"}


def _device_errors(ref, got) -> dict:
    """max |got - ref| / max |ref| per field on the device (u on the largest |u| component)."""
    r0, u0, T0 = ref
    r1, u1, T1 = got
    us = max(float(u0[a].abs().max()) for a in range(3))
    return {"rho": float((r1 - r0).abs().max() / r0.abs().max()),
            "T": float((T1 - T0).abs().max() / T0.abs().max()),
            "u": max(float((u1[a] - u0[a]).abs().max()) for a in range(3)) / us}


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1111_0905_gb300 import build, lb

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    lb.load_library()
    stream = torch.cuda.current_stream()
    peaks = measured_peaks()

    def barrier():
        if ws > 1:
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        return replica_aggregate(x, 1, 1, ws, device="cuda")[0]

    def time_steps(lat, K, W, clocks=None):
        lat.step(W)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        if clocks is not None:
            clocks.__enter__()
        e0.record(stream)
        lat.step(K)
        e1.record(stream)
        e1.synchronize()
        if clocks is not None:
            clocks.__exit__(None, None, None)
        torch.cuda.synchronize()
        barrier()
        return e0.elapsed_time(e1)

    n = args.n
    main_form = args.only or "f32"
    w_main = workload(main_form, n)
    p0 = w_main.params
    N = p0.nx * p0.ny * p0.nz
    rho_np, T_np = w_main.fields()
    rho_d = torch.from_numpy(rho_np).cuda()
    T_d = torch.from_numpy(T_np).cuda()
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        uuid = None

    results = {}
    clock_summary = None
    form_list = [args.only] if args.only else list(FORM_ORDER)
    for form in form_list:
        p = workload(form, n).params
        if args.only:
            p.nu_every = args.nu_every
        lat = lb.Lattice(p, rho_d, T_d)
        launch = lat.launch_info()
        K = args.steps if (form == main_form or form != "f64") else min(args.steps, F64_MAX_STEPS)
        sampler = ClockSampler(uuid) if form == main_form else None
        ms = time_steps(lat, K, args.warmup, sampler)
        if sampler is not None:
            clock_summary = sampler.summary()
        health = lat.diagnostics()          # outside the timed region: the state stayed physical
        lat.close()
        ms = max_over_ranks(ms)
        per_step = ms / K
        bytes_step = 4 * Q * N * STORE_BYTES[form]
        results[form] = {"glups": N / (per_step * 1e-3) / 1e9 * ws, "ms_per_step": per_step,
                         "steps": K, "warmup": args.warmup,
                         "state_after": {"min_rho": float(health["min_rho"]),
                                         "min_T": float(health["min_T"]),
                                         "nonfinite": int(health["nonfinite"])},
                         "hbm_gbs_algorithmic": bytes_step / (per_step * 1e-3) / 1e9,
                         "hbm_frac": bytes_step / (per_step * 1e-3) / 1e9 / peaks["hbm_gbs"],
                         "bytes_per_node": 4 * Q * STORE_BYTES[form],
                         "stored_bytes_per_node": 4 * STORED_SLOTS[form] * STORE_BYTES[form],
                         "launch": launch}
        torch.cuda.empty_cache()

    # the bound of the access pattern itself: the step's loads and stores without its arithmetic
    pattern = stream_bound_sweep(lb, torch, peaks, p0, results[main_form]["launch"]["ctas_per_sm"])
    for form in results:
        b = pattern.get(f"{STORE_BYTES[form]}B") if form in PATTERN_FORMS else None
        if b is not None:
            results[form]["frac_of_pattern_bound"] = results[form]["hbm_gbs_algorithmic"] / b["same_residency"]["GBs"]

    if args.only:
        if rank == 0:
            print(json.dumps({"only": args.only, "n": n, "form": results[args.only],
                              "pattern_bound": pattern}))
        if ws > 1:
            dist.destroy_process_group()
        return None

    # error of each form against the FP64 step after ERR_STEPS_HEADLINE steps of the same cell,
    # compared on the device
    ref = None
    shape = (p0.nz, p0.ny, p0.nx)
    for form in ("f64", "f32", "fp16loc", "fp16dev", "bf16dev"):
        lat = lb.Lattice(workload(form, n).params, rho_d, T_d)
        lat.step(ERR_STEPS_HEADLINE)
        outs = [torch.empty(shape, dtype=torch.float64, device="cuda") for _ in range(5)]
        lat.moments_into(*outs, device=True)
        nu = lat.nusselt()[0]
        lat.close()
        fields = (outs[0], outs[1:4], outs[4])
        if form == "f64":
            ref, nu64 = fields, nu
            results["f64"]["err_vs_f64"] = None
            results["f64"]["nu_mean_after"] = nu
        else:
            e = _device_errors(ref, fields)
            e.update({"steps": ERR_STEPS_HEADLINE, "nu_mean": nu, "nu_mean_f64": nu64,
                      "nu_rel_err": abs(nu - nu64) / abs(nu64)})
            results[form]["err_vs_f64"] = e
            del outs, fields
        torch.cuda.empty_cache()
    del ref
    torch.cuda.empty_cache()
    for form in ("f32", "fp16loc", "fp16dev", "bf16dev"):
        results[form]["speedup_vs_f64"] = results[form]["glups"] / results["f64"]["glups"]
    results["f64"]["fp64_alu"] = fp64_alu_roofline(results["f64"]["ms_per_step"], N)

    # C5 itself: 1000 timed steps of the FP32 and FP16-deviation forms at 512^3
    c5 = {}
    if not args.no_sizes and n == HEADLINE_N:
        for form in ("f32", "fp16loc", "fp16dev"):
            if form == main_form and args.steps == C5_STEPS:
                c5[form] = {"glups": results[form]["glups"], "ms_per_step": results[form]["ms_per_step"],
                            "hbm_frac": results[form]["hbm_frac"], "steps": C5_STEPS}
                continue
            lat = lb.Lattice(workload(form, n).params, rho_d, T_d)
            ms = max_over_ranks(time_steps(lat, C5_STEPS, args.warmup)) / C5_STEPS
            lat.close()
            bytes_step = 4 * Q * N * STORE_BYTES[form]
            c5[form] = {"glups": N / (ms * 1e-3) / 1e9 * ws, "ms_per_step": ms, "steps": C5_STEPS,
                        "hbm_frac": bytes_step / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"]}
            torch.cuda.empty_cache()
    del rho_d, T_d
    torch.cuda.empty_cache()

    # end to end through the C ABI with host buffers: H2D of the initial fields from pinned
    # memory, K steps, Nu and the moment fields back to pinned host memory
    p = w_main.params
    rho_h = torch.from_numpy(rho_np).pin_memory()
    T_h = torch.from_numpy(T_np).pin_memory()
    del rho_np, T_np
    outs = [torch.empty((p.nz, p.ny, p.nx), dtype=torch.float64).pin_memory() for _ in range(5)]
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    lat = lb.Lattice(p, rho_h, T_h)
    lat.step(args.steps)
    nu_mean, nu_z, _ = lat.nusselt()
    lat.moments_into(*outs, device=False)
    torch.cuda.synchronize()
    t_e2e = max_over_ranks(time.perf_counter() - t0)
    lat.close()
    e2e = {"value": N * args.steps * ws / t_e2e / 1e9, "unit": UNIT,
           "h2d_bytes_per_step": 2 * N * 8 / args.steps,
           "d2h_bytes_per_step": (5 * N * 8 + (p.nz + 1) * 8 + 16) / args.steps,
           "seconds": t_e2e, "nu_mean": nu_mean,
           "what": "lb_init from pinned host rho,T + lb_step(K) + lb_nusselt + lb_moments to "
                   "pinned host, wall clock, headline cell and form"}
    del outs, rho_h, T_h

    sizes = {} if args.no_sizes else size_sweep(args, lb, torch, peaks, max_over_ranks, barrier, ws)
    variants = {} if args.no_sizes else variant_sweep(lb, torch, peaks, max_over_ranks, barrier, ws)
    diagnostics = {} if args.no_sizes else diagnostics_cost(lb, torch, max_over_ranks, barrier, sizes)
    adjoint = {} if args.no_sizes else adjoint_cost(lb, torch)
    horizons = {} if args.no_sizes else horizon_errors(lb, torch, np)

    main = results[main_form]
    src_hash = kernel_src_hash()
    traffic = None
    if TRAFFIC["src_hash"] == src_hash:
        t = TRAFFIC["bytes_per_launch"].get(main_form)
        traffic = None if t is None else t * N / TRAFFIC["nodes"]
    bytes_launch = 4 * Q * STORE_BYTES[main_form] * N
    roofline = {"bound": "hbm", "achieved": bytes_launch / (main["ms_per_step"] * 1e-3) / 1e9,
                "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": bytes_launch / (main["ms_per_step"] * 1e-3) / 1e9 / peaks["hbm_gbs"],
                "traffic": traffic, "peak_src": peaks["src"] + " (MEASURED_PEAKS.json hbm_gbs, burst copy)",
                "traffic_src": TRAFFIC["what"] if traffic is not None else "kernel sources changed since the capture",
                "kernel": f"tlbm::lb_fused_kernel<{KERNEL_TYPE[main_form]},8,0,0>",
                "algorithmic_bytes_per_launch": bytes_launch,
                "algorithmic": f"76 values x {STORE_BYTES[main_form]} B x {N} nodes (19 f + 19 g read and written)"}
    pb = pattern.get(f"{STORE_BYTES[main_form]}B") if main_form in PATTERN_FORMS else None
    if pb is not None:
        same = pb["same_residency"]
        roofline["pattern_bound"] = {
            "GBs": same["GBs"], "frac_of_peak": same["frac_of_peak"], "warps_per_sm": same["warps_per_sm"],
            "frac_achieved_of_it": roofline["achieved"] / same["GBs"],
            "what": "lb_stream_bound (the step's 76 loads and stores per node, no arithmetic) timed live "
                    "at the fused kernel's resident warps per SM"}

    out = None
    if rank == 0:
        cpu = None if (ws > 1 or args.no_cpu_baseline) else cpu_baseline(args)
        out = {"metric": METRIC, "value": main["glups"], "unit": UNIT, "n_gpus": ws,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": main["ms_per_step"],
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
               "data": "synthetic (seeded SplitMix64 fields; no dataset)",
               "config": config_dict(w_main, main_form), "roofline": roofline, "cpu_baseline": cpu,
               "e2e": e2e, "gpu_launches": args.steps, "clocks": clock_summary,
               "forms": results, "c5_1000_steps": c5, "sizes": sizes, "variants": variants,
               "diagnostics": diagnostics, "adjoint": adjoint, "horizon_errors": horizons,
               "pattern_bound_sweep": pattern,
               "kernel_src_hash": src_hash}
        print(json.dumps(out))
    if ws > 1:
        dist.destroy_process_group()
    return out


def stream_bound_sweep(lb, torch, peaks, p, fused_ctas: int) -> dict:
    """lb_stream_bound on the cell's grid in 4- and 2-byte elements: at the fused kernel's residency
    (its CTAs per SM, 256 threads each like the fused kernel's), at the yardstick's own occupancy
    limit, and one node per thread. 76 values per node per launch; inputs far larger than L2 and
    alternated between two pairs of lattices."""
    shape = (p.nz, p.ny, p.nx)
    N = p.nx * p.ny * p.nz
    st = torch.cuda.current_stream()
    out = {}
    for elem, dt in ((4, torch.float32), (2, torch.float16)):
        bufs = [torch.zeros(Q * N, dtype=dt, device="cuda") for _ in range(4)]
        occ = lb.stream_bound(*bufs, shape, 0)
        res = {}
        for name, ctas in (("same_residency", min(fused_ctas, occ)), ("occupancy_limit", occ),
                           ("node_per_thread", 0)):
            def launch(k):
                a, b = (0, 2) if k % 2 == 0 else (2, 0)
                lb.stream_bound(bufs[a], bufs[a + 1], bufs[b], bufs[b + 1], shape, ctas)
            for k in range(3):
                launch(k)
            K = 10
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(st)
            for k in range(K):
                launch(k)
            e1.record(st)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / K
            gbs = 4 * Q * elem * N / (ms * 1e-3) / 1e9
            res[name] = {"ctas_per_sm": ctas, "warps_per_sm": 8 * ctas if ctas else None, "ms": ms,
                         "GBs": gbs, "frac_of_peak": gbs / peaks["hbm_gbs"]}
        out[f"{elem}B"] = res
        del bufs
        torch.cuda.empty_cache()
    return out


def fp64_alu_roofline(ms_per_step: float, N: int) -> dict:
    """FP64 form against GB300's FP64 pipe: FP64 operations per node (counted by ncu) x nodes per
    step / step time, against the nominal FP64 rate."""
    if FP64_FLOPS_PER_NODE is None:
        return {"bound": "alu", "achieved": None, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": None, "what": "FP64 operation count not captured for these sources"}
    achieved = FP64_FLOPS_PER_NODE * N / (ms_per_step * 1e-3) / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS, "flops_per_node": FP64_FLOPS_PER_NODE,
            "peak_src": "nominal: 152 SMs x 2 FP64 FMA/clk x 2 flops x 2.07 GHz"}


def _timed(lb, torch, max_over_ranks, barrier, p, rho, T, K, W=10):
    lat = lb.Lattice(p, torch.from_numpy(rho).cuda(), torch.from_numpy(T).cuda())
    launch = lat.launch_info()
    lat.step(W)
    torch.cuda.synchronize()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    st = torch.cuda.current_stream()
    e0.record(st)
    lat.step(K)
    e1.record(st)
    e1.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1)) / K
    health = lat.diagnostics()
    lat.close()
    torch.cuda.empty_cache()
    return ms, launch, health


def size_sweep(args, lb, torch, peaks, max_over_ranks, barrier, ws) -> dict:
    """GLUPS and HBM fraction of every form on the 128^3 single-phase convection cell and of the
    FP32 and FP16-deviation forms on the 256^3 paper-geometry boiling cell (200 timed steps
    after 10 warm-up steps; FP64 50 steps)."""
    out = {}
    for n, forms in ((128, ("f32", "fp16loc", "fp16dev", "bf16dev", "f64")), (256, ("f32", "fp16loc", "fp16dev"))):
        for form in forms:
            w = workload(form, n)
            p = w.params
            N = p.nx * p.ny * p.nz
            rho, T = w.fields()
            K = 50 if form == "f64" else 200
            ms, launch, health = _timed(lb, torch, max_over_ranks, barrier, p, rho, T, K)
            bytes_step = 4 * Q * STORE_BYTES[form] * N
            out[f"{n}^3_{form}"] = {"glups": N / (ms * 1e-3) / 1e9 * ws, "ms_per_step": ms, "steps": K,
                                    "hbm_frac": bytes_step / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
                                    "workload": describe(w), "launch": launch,
                                    "nonfinite": int(health["nonfinite"])}
    return out


def diagnostics_cost(lb, torch, max_over_ranks, barrier, sizes) -> dict:
    """Cost of sampling Nu(z) and the health values every step (nu_every = 1: the step launch
    takes the sample in passing, plus the finalisation) on the FP32 128^3 cell, 200 timed steps
    after 10 warm-up, against the same cell without samples."""
    w = workload("f32", 128)
    p = w.params
    p.nu_every = 1
    rho, T = w.fields()
    ms, _, _ = _timed(lb, torch, max_over_ranks, barrier, p, rho, T, 200)
    ms_step = sizes.get("128^3_f32", {}).get("ms_per_step")
    return {"workload": describe(w) + ", f32 form", "nu_every": 1, "ms_per_step": ms,
            "ms_per_sample": None if ms_step is None else ms - ms_step, "step_only_ms": ms_step}


def adjoint_cost(lb, torch) -> dict:
    """The discrete adjoint on the 64^3 boiling cell (FP64, 1000 steps): wall time of
    lb_adjoint_step (J and dJ/d(T_d, T_u, G)) with the segment length taken from free device
    memory (every state's fields kept: 42 GB here) and with checkpoints every 50 steps, against
    (a) the plain forward run, lb_step(1000) with no Nu sampling, and (b) the forward run that
    computes J (1000 steps with a Nu sample each, then lb_nusselt), all from lb_init's state."""
    from paper_1111_0905_gb300 import config
    w = config.boiling_cell(64, kappa=0.15, tau_nu=1.25)
    p = w.params
    rho, T = w.fields()
    N, K = 1000, 50

    def wall(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0, r

    lat = lb.Lattice(p, rho, T)
    lat.step(5)                    # warm-up of the kernels, then a fresh context for each run
    lat.close()
    lat = lb.Lattice(p, rho, T)
    t_adj, got = wall(lambda: lat.adjoint(N, 0))
    lat.close()
    torch.cuda.empty_cache()
    lat = lb.Lattice(p, rho, T)
    t_adj_k, got_k = wall(lambda: lat.adjoint(N, K))
    lat.close()
    lat = lb.Lattice(p, rho, T)
    t_plain, _ = wall(lambda: lat.step(N))
    lat.close()
    q = lb.Params(**{**p.__dict__, "nu_every": 1})
    lat = lb.Lattice(q, rho, T)
    t_fwd, J = wall(lambda: (lat.step(N), lat.nusselt()[2])[1])
    lat.close()
    return {"workload": "boiling cell 64^3 FP64, 1000 steps",
            "adjoint_s": t_adj, "segment": "from free memory (checkpoint_every = 0): all 1000 states' fields",
            "forward_plain_s": t_plain, "forward_with_J_s": t_fwd,
            "ratio_vs_plain_step": t_adj / t_plain, "ratio_vs_forward_with_J": t_adj / t_fwd,
            "checkpointed_every_50": {"adjoint_s": t_adj_k, "ratio_vs_plain_step": t_adj_k / t_plain,
                                      "ratio_vs_forward_with_J": t_adj_k / t_fwd,
                                      "grad_rel_diff": max(abs(got_k[k] - got[k]) / abs(got[k])
                                                           for k in ("T_d", "T_u", "G"))},
            "J": got["J"], "J_rel_diff_vs_forward": abs(got["J"] - J) / abs(J),
            "dJ_dTd": got["T_d"], "dJ_dTu": got["T_u"], "dJ_dG": got["G"]}


def horizon_errors(lb, torch, np) -> dict:
    """Errors of the mixed forms against the FP64 step at the stated horizons of the two
    configurations they are quoted on: the 128^3 single-phase cell after 2000 steps and the 256^3
    boiling cell after 5000 steps (FP32, FP16 against local references, BF16 and FP16 deviations).
    Field errors are max |form - FP64| / max |FP64| (u on the largest |u|), with the root mean
    square of the rho error beside it; Nu_mean of each run and the relative mass change."""
    from paper_1111_0905_gb300 import config
    out = {}
    for name, make, n, steps in (("single_phase_128^3", config.single_phase_cell, 128, 2000),
                                 ("boiling_256^3", config.paper_scale_cell, 256, 5000)):
        runs = {}
        for form in ("f64", "f32", "fp16loc", "bf16dev", "fp16dev"):
            w = make(n, precision=FORMS[form])
            rho, T = w.fields()
            lat = lb.Lattice(w.params, torch.from_numpy(rho).cuda(), torch.from_numpy(T).cuda())
            m0 = float(lat.diagnostics()["mass"])
            lat.step(steps)
            r, u, TT = lat.moments()
            h = lat.diagnostics()
            runs[form] = (r, u, TT, lat.nusselt()[0], float(h["mass"]) / m0 - 1.0, int(h["nonfinite"]))
            lat.close()
            del rho, T
            torch.cuda.empty_cache()
        r64, u64, T64, nu64, dm64, _ = runs["f64"]
        entry = {"steps": steps, "f64": {"nu_mean": nu64, "mass_change": dm64}}
        for form in ("f32", "fp16loc", "bf16dev", "fp16dev"):
            r, u, TT, nu, dm, bad = runs[form]
            entry[form] = {
                "rho": float(np.abs(r - r64).max() / np.abs(r64).max()),
                "rho_rms": float(np.sqrt(np.mean((r - r64) ** 2)) / np.abs(r64).max()),
                "T": float(np.abs(TT - T64).max() / np.abs(T64).max()),
                "u": float(max(np.abs(u[a] - u64[a]).max() for a in range(3)) /
                           max(np.abs(u64[a]).max() for a in range(3))),
                "nu_mean": nu, "nu_rel_err": float(abs(nu - nu64) / abs(nu64)),
                "mass_change": dm, "nonfinite": bad}
        out[name] = entry
    return out


def variant_sweep(lb, torch, peaks, max_over_ranks, barrier, ws) -> dict:
    """GLUPS of the scheme variants (Guo forcing, van der Waals psi) in the FP32 form on the 128^3
    single-phase cell (the van der Waals psi with its liquid, rho = 6.0 at T_m; a = 5/42,
    b = 2/21), 200 timed steps after 10 warm-up steps each, beside the paper's scheme."""
    from paper_1111_0905_gb300 import config, synthetic
    out = {}
    for name, forcing, psi in (("paper", 0, 0), ("guo", 1, 0), ("vdw", 0, 1), ("guo+vdw", 1, 1)):
        w = config.single_phase_cell(128, precision=FORMS["f32"])
        p = w.params
        p.forcing, p.psi_kind = forcing, psi
        rho, T = w.fields()
        if psi:
            p.G = -1.0
            rho, T = synthetic.single_phase_fields(p.nx, p.ny, p.nz, 6.0, p.T_d, p.T_u)
        N = p.nx * p.ny * p.nz
        lat = lb.Lattice(p, torch.from_numpy(rho).cuda(), torch.from_numpy(T).cuda())
        launch = lat.launch_info()
        lat.step(10)
        torch.cuda.synchronize()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        K = 200
        e0.record()
        lat.step(K)
        e1.record()
        e1.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1)) / K
        health = lat.diagnostics()
        lat.close()
        bytes_step = 4 * Q * STORE_BYTES["f32"] * N
        out[name] = {"glups": N / (ms * 1e-3) / 1e9 * ws, "ms_per_step": ms,
                     "hbm_frac": bytes_step / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
                     "registers": launch["registers"], "nonfinite": int(health["nonfinite"])}
    return out


def _oracle_block(side: int):
    """Oracle state and params of a side^3 block of the headline cell: the corner block on the
    bottom wall of the 512^3 paper-geometry boiling cell, with that cell's parameters (its
    gravity, conductivity, relaxation times and wall temperatures) and its own initial values at
    those nodes (drawn from the same generator counters)."""
    import torch
    from oracle import lbm
    from paper_1111_0905_gb300 import synthetic
    w = workload("f64", HEADLINE_N)
    p = w.params
    op = lbm.Params(side, side, side, p.tau_nu, p.tau_kappa, p.G, p.kappa, p.c_v, p.g_z, p.T_d, p.T_u)
    rho, T = synthetic.boiling_block(p.nx, p.ny, p.nz, 0, 0, 0, side, side, side, w.rho_mean,
                                     p.T_d, p.T_u)
    f, g = lbm.init_state(torch.from_numpy(rho), torch.from_numpy(T), op)
    return f, g, op


def cpu_baseline(args) -> dict:
    """FP64 oracle timed on the host cores on a bounded sample of the headline cell: a 128^3
    block of the 512^3 cell, as many steps as take about 15 s (6 to 100) after one warm-up step;
    then on one host thread, as many steps as take about 8 s (1 to 20)."""
    import torch
    from oracle import lbm
    side = 128
    f, g, op = _oracle_block(side)
    t0 = time.perf_counter()
    f, g = lbm.step(f, g, op)  # warm-up, also sizes the sample
    n = max(6, min(100, int(15.0 / max(time.perf_counter() - t0, 1e-3))))
    t0 = time.perf_counter()
    for _ in range(n):
        f, g = lbm.step(f, g, op)
    dt = time.perf_counter() - t0
    threads = torch.get_num_threads()
    torch.set_num_threads(1)
    try:
        t1 = time.perf_counter()
        f, g = lbm.step(f, g, op)
        n1 = max(1, min(20, int(8.0 / max(time.perf_counter() - t1, 1e-3))))
        t1 = time.perf_counter()
        for _ in range(n1):
            f, g = lbm.step(f, g, op)
        dt1 = time.perf_counter() - t1
    finally:
        torch.set_num_threads(threads)
    what = f"{side}^3 block of the {HEADLINE_N}^3 paper-geometry boiling cell (FP64 oracle, PyTorch CPU)"
    return {"value": side ** 3 * n / dt / 1e9, "unit": UNIT, "cores": threads,
            "kind": "oracle", "sample": f"{n} steps of a {what}", "seconds": dt,
            "single_thread": {"value": side ** 3 * n1 / dt1 / 1e9, "unit": UNIT, "cores": 1,
                              "sample": f"{n1} steps of the same block", "seconds": dt1}}


def run_reference(args):
    """The oracle as the reference arm: each step is one FP64 oracle step of a cube block of the
    headline cell, the cube sized so that warm-up + timed steps stay within about two minutes."""
    import torch
    from oracle import lbm
    ws, rank, local = dist_env()
    if rank != 0:
        return None
    side = 8
    for s in (32, 16, 8):
        f, g, op = _oracle_block(s)
        t0 = time.perf_counter()
        lbm.step(f, g, op)
        if (time.perf_counter() - t0) * (args.steps + args.warmup) < 120.0:
            side = s
            break
    f, g, op = _oracle_block(side)
    for _ in range(args.warmup):
        f, g = lbm.step(f, g, op)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f, g = lbm.step(f, g, op)
    dt = time.perf_counter() - t0
    nodes = side ** 3
    value = nodes * args.steps / dt / 1e9
    w = workload("f64", HEADLINE_N)
    sample = (f"each step = one FP64 oracle step of a {side}^3 block (corner on the bottom wall) of "
              f"the {HEADLINE_N}^3 cell")
    cfg = config_dict(w, "f64")
    cfg.update({"workload": f"{side}^3 block of the {describe(w)}, FP64 oracle on the host cores",
                "grid": [side, side, side], "nodes": nodes, "sample_of": [w.params.nx] * 3})
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded SplitMix64 fields; no dataset)",
           "config": cfg,
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": torch.get_num_threads(),
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=C5_STEPS)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sizes", action="store_true",
                    help="skip the extra entries (1000-step C5 timings, 128^3/256^3, variants, "
                         "diagnostics, adjoint, horizon errors)")
    ap.add_argument("--only", choices=list(FORMS), help="time one form only (no errors, e2e or "
                    "baselines; for profiling)")
    ap.add_argument("--nu-every", type=int, default=0, help="with --only: sample Nu every n steps "
                    "inside the timed steps (the diagnostics path)")
    ap.add_argument("--n", type=int, default=HEADLINE_N, choices=[128, 192, 256, 512],
                    help="cube size (default 512, the headline; 128: the single-phase convection "
                         "cell; 192/256: the boiling cell; smaller sizes for profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
