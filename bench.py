#!/usr/bin/env python
"""Benchmark of the fused thermal D3Q19 lattice Boltzmann step on GB300.

Workload: the single-phase thermal convection cell 128^3 (compressed liquid rho = 2.30 between
a hot bottom and a cold top wall, Pr = 9, seeded 1 % temperature noise), the FP32 form as the
headline, with the FP64, BF16-deviation and FP16-deviation forms of the same cell reported
beside it with their error against the FP64 step. One "step" is one full time step of the
method (pull streaming, moments, psi, force, velocities, divergence, f and g collisions, walls)
= one fused kernel launch. Value = lattice-node updates per second (GLUPS) of the whole job.

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
FORMS = {"f64": 0, "f32": 1, "bf16dev": 2, "fp16dev": 3}
STORE_BYTES = {"f64": 8, "f32": 4, "bf16dev": 2, "fp16dev": 2}
ERR_STEPS = 200

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the fused step
# kernel from an ncu capture, keyed by the hash of the kernel sources it was taken on; it is
# reported as null when the sources have changed since.
TRAFFIC = {"src_hash": "53645933b324c7a2",
           "bytes_per_launch": {"f32": 337961472 + 276750080, "fp16dev": 167004160 + 117662976}}


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


def workload(prec_name: str, n: int = 128):
    """The headline 128^3 single-phase cell, or (n > 128, profiling with --only) the
    paper-geometry boiling cell of the size sweep."""
    from paper_1111_0905_gb300 import config
    if n > 128:
        return config.paper_scale_cell(n, precision=FORMS[prec_name])
    return config.single_phase_cell(128, precision=FORMS[prec_name])


def config_dict(w, form: str) -> dict:
    p = w.params
    N = p.nx * p.ny * p.nz
    in_bytes = 2 * Q * N * STORE_BYTES[form]
    return {"workload": f"single-phase thermal convection cell {p.nx}x{p.ny}x{p.nz} "
                        f"(rho=2.30, Pr=9, tau_nu={p.tau_nu:g}, tau_kappa={p.tau_kappa:g}, "
                        f"Ra=0.5*Ra_max), {form} form",
            "grid": [p.nx, p.ny, p.nz], "nodes": N, "form": form,
            "l2": f"inputs larger than L2: {in_bytes / 1e6:.0f} MB of populations read per step "
                  f"> 129 MB L2; no flush",
            "parallelism": "replicas", "lattice": "D3Q19 x2 (f, g)"}


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
        ctx = clocks if clocks is not None else None
        if ctx is not None:
            ctx.__enter__()
        e0.record(stream)
        lat.step(K)
        e1.record(stream)
        e1.synchronize()
        if ctx is not None:
            ctx.__exit__(None, None, None)
        torch.cuda.synchronize()
        barrier()
        return e0.elapsed_time(e1)

    results = {}
    fields = {}
    main_form = "f32"
    clock_summary = None
    form_list = [args.only] if args.only else ["f32", "f64", "bf16dev", "fp16dev"]
    for form in form_list:
        w = workload(form, args.n if args.only else 128)
        p = w.params
        if args.only:
            p.nu_every = args.nu_every
        N = p.nx * p.ny * p.nz
        rho, T = w.fields()
        rho_d = torch.from_numpy(rho).cuda()
        T_d = torch.from_numpy(T).cuda()
        lat = lb.Lattice(p, rho_d, T_d)
        launch = lat.launch_info()
        K = args.steps if form == main_form else min(args.steps, 2000)
        W = args.warmup
        uuid = None
        try:
            uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
        except Exception:
            uuid = None
        sampler = ClockSampler(uuid) if form == main_form else None
        ms = time_steps(lat, K, W, sampler)
        if sampler is not None:
            clock_summary = sampler.summary()
        health = lat.diagnostics()          # outside the timed region: the state stayed physical
        ms = max_over_ranks(ms)
        per_step = ms / K
        lat.close()
        # error of this form against the FP64 step after ERR_STEPS steps of the same cell
        lat = lb.Lattice(p, rho_d, T_d)
        lat.step(ERR_STEPS)
        r, u, TT = lat.moments()
        nu = lat.nusselt()[0]
        lat.close()
        fields[form] = (r, u, TT, nu)
        bytes_step = 2 * 2 * Q * N * STORE_BYTES[form]
        glups_rank = N / (per_step * 1e-3) / 1e9
        results[form] = {"glups": glups_rank * ws, "ms_per_step": per_step, "steps": K,
                         "state_after": {"min_rho": float(health["min_rho"]),
                                         "min_T": float(health["min_T"]),
                                         "nonfinite": int(health["nonfinite"])},
                         "hbm_gbs_algorithmic": bytes_step / (per_step * 1e-3) / 1e9,
                         "hbm_frac": bytes_step / (per_step * 1e-3) / 1e9 / peaks["hbm_gbs"],
                         "bytes_per_node": 4 * Q * STORE_BYTES[form], "launch": launch}
        del rho_d, T_d
        torch.cuda.empty_cache()

    if args.only:
        if rank == 0:
            print(json.dumps({"only": args.only, "form": results[args.only]}))
        if ws > 1:
            dist.destroy_process_group()
        return None
    r64, u64, T64, nu64 = fields["f64"]
    for form, (r, u, TT, nu) in fields.items():
        results[form]["err_vs_f64"] = None if form == "f64" else {
            "steps": ERR_STEPS,
            "rho": float(np.abs(r - r64).max() / np.abs(r64).max()),
            "T": float(np.abs(TT - T64).max() / np.abs(T64).max()),
            "u": float(max(np.abs(u[a] - u64[a]).max() for a in range(3)) /
                       max(np.abs(u64[a]).max() for a in range(3))),
            "nu_mean": float(abs(nu - nu64) / max(abs(nu64), 1e-300))}

    # end to end through the C ABI with host buffers: H2D of the initial fields from pinned
    # memory, K steps, Nu and the moment fields back to pinned host memory
    w = workload(main_form)
    p = w.params
    N = p.nx * p.ny * p.nz
    rho, T = w.fields()
    rho_h = torch.from_numpy(rho).pin_memory()
    T_h = torch.from_numpy(T).pin_memory()
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
           "what": "lb_init from pinned host rho,T + lb_step(K) + lb_nusselt + lb_moments to "
                   "pinned host, wall clock"}

    # the sizes the HBM target is stated at (256^3, 512^3), same kernel, paper-geometry boiling cell
    sizes = {} if args.no_sizes else size_sweep(args, lb, torch, peaks, max_over_ranks, barrier, ws)
    variants = {} if args.no_sizes else variant_sweep(lb, torch, peaks, max_over_ranks, barrier, ws)
    diagnostics = diagnostics_cost(lb, torch, max_over_ranks, barrier, results[main_form]["ms_per_step"])
    adjoint = {} if args.no_sizes else adjoint_cost(lb, torch)
    horizons = {} if args.no_sizes else horizon_errors(lb, torch, np)

    main = results[main_form]
    src_hash = kernel_src_hash()
    traffic = None
    if TRAFFIC["src_hash"] == src_hash:
        traffic = TRAFFIC["bytes_per_launch"].get(main_form)
    bytes_launch = 4 * Q * STORE_BYTES[main_form] * N
    roofline = {"bound": "hbm", "achieved": bytes_launch / (main["ms_per_step"] * 1e-3) / 1e9,
                "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": bytes_launch / (main["ms_per_step"] * 1e-3) / 1e9 / peaks["hbm_gbs"],
                "traffic": traffic, "peak_src": peaks["src"] + " (MEASURED_PEAKS.json hbm_gbs)",
                "kernel": "tlbm::lb_fused_kernel<float,8,0>", "algorithmic_bytes_per_launch": bytes_launch}

    out = None
    if rank == 0:
        cpu = None if (ws > 1 or args.no_cpu_baseline) else cpu_baseline(args)
        out = {"metric": METRIC, "value": main["glups"], "unit": UNIT, "n_gpus": ws,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": main["ms_per_step"],
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
               "data": "synthetic (seeded SplitMix64 fields; no dataset)",
               "config": config_dict(w, main_form), "roofline": roofline, "cpu_baseline": cpu,
               "e2e": e2e, "gpu_launches": args.steps, "clocks": clock_summary,
               "forms": results, "sizes": sizes, "variants": variants, "diagnostics": diagnostics,
               "adjoint": adjoint, "horizon_errors": horizons,
               "kernel_src_hash": src_hash}
        print(json.dumps(out))
    if ws > 1:
        dist.destroy_process_group()
    return out


def size_sweep(args, lb, torch, peaks, max_over_ranks, barrier, ws) -> dict:
    """GLUPS and HBM fraction of the FP32 and FP16-deviation forms on the boiling cell at 256^3
    and 512^3 (50 timed steps after 10 warm-up steps each)."""
    from paper_1111_0905_gb300 import config
    out = {}
    for n in (256, 512):
        for form in ("f32", "fp16dev"):
            w = config.paper_scale_cell(n, precision=FORMS[form])
            p = w.params
            N = p.nx * p.ny * p.nz
            rho, T = w.fields()
            lat = lb.Lattice(p, torch.from_numpy(rho).cuda(), torch.from_numpy(T).cuda())
            launch = lat.launch_info()
            del rho, T
            lat.step(10)
            torch.cuda.synchronize()
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            K = 50
            e0.record()
            lat.step(K)
            e1.record()
            e1.synchronize()
            ms = max_over_ranks(e0.elapsed_time(e1)) / K
            lat.close()
            torch.cuda.empty_cache()
            bytes_step = 4 * Q * STORE_BYTES[form] * N
            out[f"{n}^3_{form}"] = {"glups": N / (ms * 1e-3) / 1e9 * ws, "ms_per_step": ms,
                                    "hbm_frac": bytes_step / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
                                    "workload": w.name, "launch": launch}
    return out


def diagnostics_cost(lb, torch, max_over_ranks, barrier, ms_step: float) -> dict:
    """Cost of sampling Nu(z) and the health values every step (nu_every = 1: one moments pass
    and one finalisation per step) on the FP32 128^3 cell, 200 timed steps after 10 warm-up."""
    w = workload("f32")
    p = w.params
    p.nu_every = 1
    rho, T = w.fields()
    lat = lb.Lattice(p, torch.from_numpy(rho).cuda(), torch.from_numpy(T).cuda())
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
    lat.close()
    return {"nu_every": 1, "ms_per_step": ms, "ms_per_sample": ms - ms_step,
            "step_only_ms": ms_step}


def adjoint_cost(lb, torch) -> dict:
    """The discrete adjoint on the 64^3 boiling cell (FP64, 1000 steps, checkpoints every 50):
    wall time of lb_adjoint_step (J and dJ/d(T_d, T_u, G)) against the forward run that computes
    J (1000 steps with a Nu sample each, then lb_nusselt), both from lb_init's state."""
    from paper_1111_0905_gb300 import config
    w = config.boiling_cell(64, kappa=0.15, tau_nu=1.25)
    p = w.params
    rho, T = w.fields()
    N, K = 1000, 50
    lat = lb.Lattice(p, rho, T)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    got = lat.adjoint(N, K)
    torch.cuda.synchronize()
    t_adj = time.perf_counter() - t0
    lat.close()
    q = lb.Params(**{**p.__dict__, "nu_every": 1})
    lat = lb.Lattice(q, rho, T)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lat.step(N)
    J = lat.nusselt()[2]
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    lat.close()
    return {"workload": "boiling cell 64^3 FP64, 1000 steps, checkpoints every 50",
            "adjoint_s": t_adj, "forward_s": t_fwd, "ratio": t_adj / t_fwd,
            "J": got["J"], "J_rel_diff_vs_forward": abs(got["J"] - J) / abs(J),
            "dJ_dTd": got["T_d"], "dJ_dTu": got["T_u"], "dJ_dG": got["G"]}


def horizon_errors(lb, torch, np) -> dict:
    """Errors of the mixed forms against the FP64 step at the stated horizons of the two
    configurations they are quoted on: the 128^3 single-phase cell after 2000 steps (FP32, BF16,
    FP16 deviations) and the 256^3 boiling cell after 5000 steps (FP32, BF16, FP16 deviations).
    Field errors are max |form - FP64| / max |FP64| (u on the largest |u|), with the root mean
    square of the rho error beside it; Nu_mean of each run and the relative mass change."""
    from paper_1111_0905_gb300 import config
    out = {}
    for name, make, n, steps in (("single_phase_128^3", config.single_phase_cell, 128, 2000),
                                 ("boiling_256^3", config.paper_scale_cell, 256, 5000)):
        runs = {}
        for form in ("f64", "f32", "bf16dev", "fp16dev"):
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
        for form in ("f32", "bf16dev", "fp16dev"):
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


def _oracle_sample(side: int):
    """Oracle state and params of a side^3 sample of the benchmark cell."""
    import torch
    from oracle import lbm
    from paper_1111_0905_gb300 import config
    w = config.single_phase_cell(128)
    p = w.params
    op = lbm.Params(side, side, side, p.tau_nu, p.tau_kappa, p.G, p.kappa, p.c_v, p.g_z, p.T_d, p.T_u)
    from paper_1111_0905_gb300 import synthetic
    rho, T = synthetic.single_phase_fields(side, side, side, 2.30, p.T_d, p.T_u)
    f, g = lbm.init_state(torch.from_numpy(rho), torch.from_numpy(T), op)
    return f, g, op


def cpu_baseline(args) -> dict:
    """FP64 oracle timed on the host cores on a bounded sample of the full 128^3 cell: as many
    steps as take about 15 s (6 to 100), after one warm-up step; then on one host thread, as many
    steps as take about 8 s (1 to 20)."""
    import torch
    from oracle import lbm
    f, g, op = _oracle_sample(128)
    t0 = time.perf_counter()
    f, g = lbm.step(f, g, op)  # warm-up, also sizes the sample
    n = max(6, min(100, int(15.0 / max(time.perf_counter() - t0, 1e-3))))
    t0 = time.perf_counter()
    for _ in range(n):
        f, g = lbm.step(f, g, op)
    dt = time.perf_counter() - t0
    # the same oracle on one host thread (a few steps of the same cell)
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
    return {"value": 128 ** 3 * n / dt / 1e9, "unit": UNIT, "cores": threads,
            "kind": "oracle", "sample": f"{n} steps of the 128^3 cell (FP64 oracle, PyTorch CPU)",
            "seconds": dt,
            "single_thread": {"value": 128 ** 3 * n1 / dt1 / 1e9, "unit": UNIT, "cores": 1,
                              "sample": f"{n1} steps of the 128^3 cell", "seconds": dt1}}


def run_reference(args):
    """The oracle as the reference arm: each step is one oracle step of a cube sample of the
    benchmark cell, the cube sized so that warm-up + timed steps stay within about two minutes."""
    import torch
    from oracle import lbm
    ws, rank, local = dist_env()
    if rank != 0:
        return None
    side = 8
    for s in (32, 16, 8):
        f, g, op = _oracle_sample(s)
        t0 = time.perf_counter()
        lbm.step(f, g, op)
        if (time.perf_counter() - t0) * (args.steps + args.warmup) < 120.0:
            side = s
            break
    f, g, op = _oracle_sample(side)
    for _ in range(args.warmup):
        f, g = lbm.step(f, g, op)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f, g = lbm.step(f, g, op)
    dt = time.perf_counter() - t0
    nodes = side ** 3
    value = nodes * args.steps / dt / 1e9
    from paper_1111_0905_gb300 import config
    w = config.single_phase_cell(128, precision=1)
    sample = f"each step = one FP64 oracle step of a {side}^3 sample of the 128^3 cell"
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded SplitMix64 fields; no dataset)",
           "config": config_dict(w, "f32"),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": torch.get_num_threads(),
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sizes", action="store_true", help="skip the 256^3/512^3 measurements")
    ap.add_argument("--only", choices=list(FORMS), help="time one form of the 128^3 cell only "
                    "(no errors, e2e or baselines; for profiling)")
    ap.add_argument("--nu-every", type=int, default=0, help="with --only: sample Nu every n steps "
                    "inside the timed steps (the diagnostics path)")
    ap.add_argument("--n", type=int, default=128, choices=[128, 256, 512],
                    help="with --only: cube size (256/512: the boiling cell of the size sweep)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
