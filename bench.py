#!/usr/bin/env python
"""MBE(3)-OSV-MP2 throughput on GB300: fragments/s of the whole pair-solve path.

One step = the full hot path over one synthetic system: OSV build (A0), OSV
projection and pair blocks (A1-A2), preconditioners (A3), the persistent
fragment solve (A4) and the MBE(3) energy (A5) -- and, with --grad, the
frozen-OSV adjoint (A6).  Workload (default): 128 occupied LMOs, 640 virtuals,
2400 auxiliary functions, envelope length 1 A, l_osv = 1e-4, pairs within 8 A
and triples within 6 A; B is regenerated on the device from its seed (never
stored) unless --b-mode stored.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

R2_CUT, R3_CUT, L_OSV = 8.0, 6.0, 1e-4
# Denominators the peaks file does not carry, measured on this GB300 pool with
# `python bench.py --measure-peaks` (torch GEMMs at 8192^3, best of 10, CUDA
# events); the figures and the run are in profiles/peaks_fp64_tf32_fp32.md.
MEASURED_GEMM_PEAKS = {"fp64_tflops": 1.099, "tf32_tflops": 1037.8, "fp32_tflops": 69.86,
                       "source": "torch.matmul 8192^3 on a GB300 of this pool, best of 10"}
FP32_SIMT_PEAK = 152 * 128 * 2 * 2.070e9 / 1e12    # 128 FFMA/clk/SM at the 2070 MHz maximum -> 80.5
# dram__bytes_read.sum + dram__bytes_write.sum per launch of the dominant kernel,
# from one single-pass ncu capture of the bench workload
# (profiles/traffic_k_eig_osv_mbe3_n128.md); kernels without a capture of their
# current code report null.
KERNEL_TRAFFIC = {"k_eig_osv": 34.27e9 + 43.22e9,          # 128-orbital workload itself (1 pass), bytes per launch
                  "k_frag_solve_mixed": 20.24e9 + 12.24e9}   # the autotuner's plan (2 CTAs per SM)


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "_fallback": True}


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            p = [x.strip() for x in l.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for k, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(k)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def fragment_energies(ctx):
    """{orbital tuple: E_C} of the ctx's last MBE(3) call."""
    orbs, _, e = ctx.fragment_results()
    return {tuple(int(x) for x in o if x >= 0): float(v) for o, v in zip(orbs, e)}


def projection_flops(ctx, s, n_osv):
    """Algorithmic A1 work of one step: B~_i^(x) = B_i^T Q_x for every x in
    dom(i) = {i} + the kept pair partners of i, i.e. 2 n_aux n_vir N_i per
    orbital with N_i = sum of n_x over dom(i) (Eq. osv_imua)."""
    orbs, _, _ = ctx.fragment_results()
    dom = [{i} for i in range(s.n_occ)]
    for o in orbs:
        if o[1] >= 0 and o[2] < 0:
            dom[o[0]].add(int(o[1]))
            dom[o[1]].add(int(o[0]))
    return sum(2.0 * s.n_aux * s.n_vir * sum(int(n_osv[x]) for x in d) for d in dom)


def measure_peaks():
    """FP64, TF32 and FP32 (no TF32) GEMM throughput with torch at 8192^3: the
    denominators of the FP64, split-TF32 and FP32 rooflines."""
    import torch
    dev = torch.device("cuda:0")
    n = 8192
    out = {}
    for name, dt, tf32 in (("fp64_tflops", torch.float64, False), ("tf32_tflops", torch.float32, True),
                           ("fp32_tflops", torch.float32, False), ("bf16_tflops", torch.bfloat16, False)):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        a = torch.randn(n, n, device=dev, dtype=dt)
        b = torch.randn(n, n, device=dev, dtype=dt)
        c = a @ b
        best = 1e30
        for _ in range(10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b, out=c)
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        out[name] = 2.0 * n ** 3 / best / 1e12
        del a, b, c
        torch.cuda.empty_cache()
    torch.backends.cuda.matmul.allow_tf32 = False
    out["how"] = "torch.matmul 8192^3, best of 10, CUDA events; tf32 = float32 with allow_tf32"
    out["gpu"] = torch.cuda.get_device_name(0)
    return out


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def job_rate(t_local, units_local, world, device="cpu"):
    """Whole-job rate of independent replicas: (units of all ranks, the slowest rank's time,
    units / time).  Every rank calls it (two all-reduces when world > 1)."""
    t, units = float(t_local), float(units_local)
    if world > 1:
        import torch
        import torch.distributed as dist
        tt = torch.tensor([t], dtype=torch.float64, device=device)
        uu = torch.tensor([units], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        dist.all_reduce(uu, op=dist.ReduceOp.SUM)
        t, units = float(tt.item()), float(uu.item())
    return units, t, units / t


# ------------------------------------------------------------------ GPU arm
def run_gpu(args):
    import torch
    import paper_2603_16575_gb300 as pkg

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    # every rank solves its own independent system (weak scaling, no data-path collective)
    s = synth.workload(args.workload, seed=args.seed + rank)
    stream = torch.cuda.Stream(dev)
    peaks = load_peaks()
    with torch.cuda.stream(stream):
        env = torch.tensor(s.env, device=dev)
        f_occ = torch.tensor(s.f_occ, device=dev)
        e_vir = torch.tensor(s.e_vir, device=dev)
        B = None
        if args.b_mode == "stored":
            B = pkg.generate_B(s.n_occ, s.n_vir, s.n_aux, s.seed, env, stream=stream.cuda_stream)
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > 129 MB L2
    stream.synchronize()
    osv_prec = "mixed" if args.prec == "mixed" else "fp64"
    ctx = pkg.Context(local, stream=stream, osv_prec=osv_prec, osv_method=args.osv_method)

    if args.osv_only:
        return run_osv_only(args, ctx, s, env, f_occ, e_vir, stream, flush, dev, pkg, torch)

    def step(B_in=B, env_in=env, f_in=f_occ, e_in=e_vir):
        kw = dict(B=B_in) if B_in is not None else dict(env=env_in, seed=s.seed, n_aux=s.n_aux)
        n_osv = ctx.build_osv(f_in, e_in, L_OSV, r_occ=s.r_occ, **kw)
        if args.grad and args.relaxed:
            E, dB, df, de, st, _ = ctx.energy_grad_relaxed(R2_CUT, R3_CUT)
        elif args.grad:
            E, dB, df, de, st = ctx.energy_grad(R2_CUT, R3_CUT, args.prec)
        elif args.screen:
            E, _, st = ctx.mbe3_energy_screened(args.prec)
        else:
            E, st = ctx.mbe3_energy(R2_CUT, R3_CUT, args.prec)
        return E, st, n_osv

    for _ in range(args.warmup):
        E, st, n_osv = step()
    grad_check = None
    if args.grad and rank == 0 and not args.no_cpu_baseline:
        # dE/dB of orbital 0 gets contributions only from the fragments containing it, so
        # the oracle checks those rows exactly from a small sample of fragments
        if args.relaxed:
            _, dB, df, de, _, gap = ctx.energy_grad_relaxed(R2_CUT, R3_CUT)
        else:
            _, dB, df, de, _ = ctx.energy_grad(R2_CUT, R3_CUT, args.prec)
        grad_check = gradient_vs_oracle(s, dB[0].cpu().numpy(), osv_method=args.osv_method, relaxed=args.relaxed)
        if args.relaxed:
            grad_check["min_gap_at_osv_cut"] = gap
        del dB, df, de
    n_frag = int(st["n_single"] + st["n_pair"] + st["n_triple"])
    ctx.profile(reset=True)
    launches0 = pkg.osvmp2.kernel_launches()
    t_steps = []
    with ClockSampler(local) as clk:
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()                       # evict L2 between timed steps (untimed)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            E, st, n_osv = step()
            ev1.record(stream)
            ev1.synchronize()
            t_steps.append(ev0.elapsed_time(ev1) / 1e3)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
    launches = pkg.osvmp2.kernel_launches() - launches0
    prof = ctx.profile(reset=True)
    gpu_frag_e = {("fp64_form" if args.prec == "fp64" else "mixed_form"): fragment_energies(ctx)}
    plan = ctx.solve_plan() if args.prec == "mixed" else None
    a0_ms = sum(prof.get(k, (0.0,))[0] for k in ("tii", "eig")) / args.steps
    # A3-A5: preconditioner, fragment solve (its set-up included) and the weighted sum
    a35_ms = sum(prof.get(k, (0.0,))[0] for k in ("precond", "solve", "mbe_sum")) / args.steps
    err = None
    if args.prec == "mixed":
        # the same inputs through the FP64 form, one step timed the same way (parity
        # of the FP64 form with the FP64 oracle is a GPU test)
        ctx.set_opts(osv_prec="fp64")
        kw = dict(B=B) if B is not None else dict(env=env, seed=s.seed, n_aux=s.n_aux)
        with torch.cuda.stream(stream):
            flush.zero_()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        ctx.build_osv(f_occ, e_vir, L_OSV, r_occ=s.r_occ, **kw)
        E64 = (ctx.mbe3_energy_screened("fp64")[0] if args.screen else ctx.mbe3_energy(R2_CUT, R3_CUT, "fp64")[0])
        ev1.record(stream)
        ev1.synchronize()
        gpu_frag_e["fp64_form"] = fragment_energies(ctx)
        t64 = ev0.elapsed_time(ev1) / 1e3
        err = {"energy_fp64_form": E64, "abs_err_eh": abs(E - E64), "rel_err": abs(E - E64) / abs(E64),
               "fp64_form_ms_per_step": 1e3 * t64, "fp64_form_fragments_per_s": n_frag / t64}
        ctx.set_opts(osv_prec=osv_prec)
        ctx.profile(reset=True)
    _, t_tot, value = job_rate(sum(t_steps), n_frag * args.steps, world, dev)

    # ---- end to end: host (pinned) inputs copied in and the energy read back every step
    pin = lambda a: torch.tensor(a).pin_memory()
    h_env, h_f, h_e = pin(s.env), pin(s.f_occ), pin(s.e_vir)
    h_B = B.cpu().pin_memory() if B is not None else None
    d_env, d_f, d_e = torch.empty_like(env), torch.empty_like(f_occ), torch.empty_like(e_vir)
    d_B = torch.empty_like(B) if B is not None else None
    h2d = sum(x.numel() * 8 for x in (h_env, h_f, h_e)) + (h_B.numel() * 8 if h_B is not None else 0)
    e2e_t = []
    for _ in range(max(1, args.steps)):
        with torch.cuda.stream(stream):
            flush.zero_()
        stream.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            d_env.copy_(h_env, non_blocking=True)
            d_f.copy_(h_f, non_blocking=True)
            d_e.copy_(h_e, non_blocking=True)
            if h_B is not None:
                d_B.copy_(h_B, non_blocking=True)
        E2, _, _ = step(B_in=d_B, env_in=d_env, f_in=d_f, e_in=d_e)   # E2 is read back to the host
        e2e_t.append(time.perf_counter() - t0)
    _, _, e2e_value = job_rate(statistics.median(e2e_t), n_frag, world, dev)

    # ---- roofline of the dominant kernel (largest device time in the timed region)
    gemm = MEASURED_GEMM_PEAKS
    peak_fp64 = gemm["fp64_tflops"]
    peak_fp32 = gemm["fp32_tflops"] or FP32_SIMT_PEAK
    peak_split = gemm["tf32_tflops"] / 10.0       # split-TF32: 10 TF32 slice products per product
    a1_flops = projection_flops(ctx, s, n_osv) * args.steps   # algorithmic A1: 2 n_aux n_vir N_i per orbital
    kern = {
        # phase key: (kernel, bound, peak TFLOP/s, peak source, algorithmic flops in the timed region)
        "k_eig": ("k_eig_osv", "alu",
                  peak_fp32 / 16.0 if args.prec == "mixed" else peak_fp64,
                  ("double-float on the FP32 pipes: FP32 peak / 16 instructions per double-float FMA"
                   if args.prec == "mixed" else "FP64 DGEMM measured"),
                  prof.get("k_eig", (0, 0))[1]),
        "k_gproj": ("k_tf32x3<EpiG2>", "tensor", peak_split,
                    f"split-TF32 on tcgen05: measured TF32 {gemm['tf32_tflops']:.0f} TF/s / 10 slice products",
                    a1_flops),
        "k_fragsolve": ("k_frag_solve_mixed" if args.prec == "mixed" else "k_frag_solve", "alu",
                        peak_fp32 if args.prec == "mixed" else peak_fp64,
                        "FP32 SIMT" if args.prec == "mixed" else "FP64 DGEMM measured",
                        prof.get("k_fragsolve", (0, 0))[1]),
    }
    kernels = {}
    for key, (kname, bound, peak, src, alg) in kern.items():
        if key not in prof or prof[key][0] <= 0:
            continue
        ms, fl, _, calls = prof[key]
        per_launch_s = ms / 1e3 / max(calls, 1)
        achieved = alg / max(calls, 1) / per_launch_s / 1e12 if alg else None
        kernels[kname] = {"phase": key, "ms_per_step": ms / args.steps, "launches_per_step": calls / args.steps,
                          "bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                          "frac": (achieved / peak) if achieved else None, "peak_source": src + " (of measured)",
                          "algorithmic_flops_per_step": alg / args.steps,
                          "performed_flops_per_step": fl / args.steps}
    dom = max(kernels.items(), key=lambda kv: kv[1]["ms_per_step"])
    dname, d = dom
    tr = KERNEL_TRAFFIC.get(dname) if (args.workload == "mbe3_n128" and args.osv_method == "exact" and
                                       args.prec == "mixed") else None
    roof = {"kernel": dname, "bound": d["bound"], "achieved": d["achieved"], "peak": d["peak"], "unit": "TFLOP/s",
            "frac": d["frac"], "traffic": tr, "peak_source": d["peak_source"],
            "per_launch": "algorithmic flops per launch / CUDA-event time per launch (library stream)"}
    top = ("tii", "eig", "sf", "project", "exchange", "precond", "solve")
    phases = {}
    alg_total = 0.0
    for k, v in prof.items():
        fl = a1_flops if (k == "project" and args.prec == "mixed") else v[1]
        if k in top:
            alg_total += fl
        tf = (fl / (v[0] / 1e3) / 1e12) if v[0] > 0 and fl else None
        phases[k] = {"ms_per_step": v[0] / args.steps, "tflops": tf}
    effective = {"value": alg_total / t_tot / 1e12 if t_tot > 0 else None, "unit": "TFLOP/s",
                 "counted": "A0 T_ii + eig, A1 projection (2 n_aux n_vir N_i per orbital), A2 K/S/F, "
                            "A3, A4 solver operations, per step"}
    if args.prec == "mixed":
        effective["projection_overhead"] = prof.get("project", (0, 0))[1] / max(a1_flops, 1.0)

    out = {
        "metric": "MBE(3) fragments/s",
        "value": value,
        "unit": "fragments/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * t_tot / args.steps,
        "step_ms": {"best": 1e3 * min(t_steps), "median": 1e3 * statistics.median(t_steps)},
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if args.prec == "fp64" else "split-tf32+f32+f64",
        "data": "synthetic",
        "config": {"workload": f"{args.workload} (n_occ={s.n_occ}, n_vir={s.n_vir}, n_aux={s.n_aux}, "
                               f"lambda={s.lam} A, l_osv={L_OSV}, " +
                               ("s2b/s3b screening 1e-7/1e-2/0.2 with weak pairs)" if args.screen
                                else f"r2={R2_CUT} A, r3={R3_CUT} A)"),
                   "prec": args.prec, "b_mode": args.b_mode, "grad": bool(args.grad),
                   "osv_relaxed": bool(args.grad and args.relaxed),
                   "osv_method": args.osv_method, "n_weak": int(st.get("n_weak", 0)),
                   "fragments": n_frag, "n_single": int(st["n_single"]), "n_pair": int(st["n_pair"]),
                   "n_triple": int(st["n_triple"]), "n_osv_mean": float(np.mean(n_osv)),
                   "l2": "256 MB buffer written between timed steps", "parallelism": f"replicas x{world}",
                   "solve_plan": plan},
        "energy": E,
        "energy_vs_fp64_form": err,
        "fragments_per_s_excl_osv_build": world * n_frag / max(1e-9, t_tot / args.steps - a0_ms / 1e3),
        "fragments_per_s_solve_only": world * n_frag / max(1e-9, a35_ms / 1e3),
        "e2e": {"value": e2e_value, "unit": "fragments/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": 8},
        "gpu_launches": int(launches),
        "gradient_vs_oracle": grad_check,
        "roofline": roof,
        "kernels": kernels,
        "effective_tflops": effective,
        "phases": phases,
        "clocks": clk.summary(),
    }
    # ---- occupied-orbital localization (Algorithm 2) on a 128-orbital synthetic set,
    # outside the timed step: its own time and rotation rate
    ls = synth.make_loc_system(s.n_occ if s.n_occ <= 256 else 128, seed=args.seed)
    Cl = torch.tensor(ls.C, dtype=torch.float64, device=dev)
    with torch.cuda.stream(stream):
        ctx.localize_pm(Cl, ls.atom_ao)           # warm-up
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        _, L_loc, sw = ctx.localize_pm(Cl, ls.atom_ao)
        ev1.record(stream)
    ev1.synchronize()
    t_loc = ev0.elapsed_time(ev1) / 1e3
    n_l = ls.C.shape[1]
    out["localization"] = {"n_occ": n_l, "n_atom": len(ls.atom_ao) - 1, "n_ao": ls.C.shape[0], "l_loc": 1e-3,
                           "sweeps": sw, "ms": 1e3 * t_loc, "functional": L_loc,
                           "pair_rotations_per_s": sw * n_l * (n_l - 1) / 2 / t_loc}
    # ---- the 20-orbital untruncated system (n_vir = 100, n_aux = 400): the full
    # osvmp2_solve over every pair in FP64, outside the timed step
    sc = synth.workload("canonical_n20", seed=args.seed)
    ctx20 = pkg.Context(local, stream=stream)
    with torch.cuda.stream(stream):
        a20 = [torch.tensor(x, device=dev) for x in (sc.f_occ, sc.e_vir, sc.env)]
        ctx20.build_osv(a20[0], a20[1], 0.0, env=a20[2], seed=sc.seed, n_aux=sc.n_aux, r_occ=sc.r_occ)
        ctx20.solve(range(sc.n_occ))                 # warm-up (pair blocks, preconditioners)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        E20, _, it20 = ctx20.solve(range(sc.n_occ))
        ev1.record(stream)
    ev1.synchronize()
    out["full_solve_n20"] = {"workload": "20 orbitals, 100 virtuals, 400 aux, untruncated (pair order 200)",
                             "energy": E20, "iterations": it20, "ms": ev0.elapsed_time(ev1),
                             "pairs": sc.n_occ * (sc.n_occ + 1) // 2}
    ctx20.close()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        e_cf = oracle.canonical_mp2_energy(sc.B_block, sc.n_occ, sc.f_occ, sc.e_vir)
        out["full_solve_n20"]["abs_err_vs_closed_form_eh"] = abs(E20 - e_cf)
        out["cpu_baseline"], ref_e = cpu_baseline(args, budget_s=args.cpu_budget)
        out["energy_vs_oracle"] = {}
        for form, got in gpu_frag_e.items():
            errs = [(abs(got[o] - e), abs(got[o] - e) / abs(e)) for o, e in ref_e.items() if o in got]
            if errs:
                out["energy_vs_oracle"][form] = {"fragments": len(errs), "max_abs_eh": max(a for a, _ in errs),
                                                 "max_rel": max(r for _, r in errs),
                                                 "sample": "fragments of the oracle CPU sample"}
    if rank == 0:
        print(json.dumps(out), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


# ------------------------------------------------------------------ CPU oracle
def cpu_sample(args, budget_s: float):
    """Oracle on a bounded sample: the k orbitals nearest to orbital 0 and every
    fragment of the workload's MBE(3) list whose orbitals all lie in that set
    (OSV build of those orbitals + all their fragment solves)."""
    import oracle
    s = synth.workload(args.workload, seed=args.seed)
    d = np.linalg.norm(s.r_occ - s.r_occ[0], axis=1)
    k = args.cpu_orbitals
    near = sorted(np.argsort(d, kind="stable")[:k].tolist())
    sel = set(near)
    frags = [(o, c) for o, c in oracle.mbe3_fragments(s.r_occ, R2_CUT, R3_CUT) if set(o) <= sel]
    t0 = time.perf_counter()
    if args.osv_method == "randomized":
        osys = oracle.OSVSystem(s.B_block, s.n_occ, s.e_vir, s.f_occ, l_osv=L_OSV, orbitals=[])
        gauss = lambda i, k: synth.gauss_row(s.seed, i, k, s.n_vir)
        osys.Q, osys.omega, _ = oracle.build_osv_randomized(osys.B, s.n_occ, s.e_vir, s.f_occ, L_OSV, gauss,
                                                            orbitals=near)
    else:
        osys = oracle.OSVSystem(s.B_block, s.n_occ, s.e_vir, s.f_occ, l_osv=L_OSV, orbitals=near)
    done = 0
    energies = {}
    for orbs, c in frags:
        energies[tuple(orbs)] = osys.solve(orbs).energy
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return done, dt, k, energies


def run_osv_only(args, ctx, s, env, f_occ, e_vir, stream, flush, dev, pkg, torch):
    """A0 alone (T_ii and the OSVs of every orbital, B regenerated on the device):
    orbitals/s, for workloads whose pair steps are out of reach (the 800-orbital
    chain).  With the CPU leg on, the OSVs of two orbitals are checked against the
    oracle with the same OSV rule."""
    def step():
        return ctx.build_osv(f_occ, e_vir, L_OSV, env=env, seed=s.seed, n_aux=s.n_aux, r_occ=s.r_occ)
    for _ in range(args.warmup):
        n_osv = step()
    ctx.profile(reset=True)
    launches0 = pkg.osvmp2.kernel_launches()
    t_steps = []
    with ClockSampler(0) as clk:
        torch.cuda.synchronize()
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            n_osv = step()
            ev1.record(stream)
            ev1.synchronize()
            t_steps.append(ev0.elapsed_time(ev1) / 1e3)
    prof = ctx.profile(reset=True)
    t_tot = sum(t_steps)
    out = {"metric": "OSV build orbitals/s", "value": s.n_occ * args.steps / t_tot, "unit": "orbitals/s",
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_tot / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "split-tf32+f64" if args.prec == "mixed" else "f64", "data": "synthetic",
           "config": {"workload": f"{args.workload} (n_occ={s.n_occ}, n_vir={s.n_vir}, n_aux={s.n_aux}, "
                                  f"{s.geometry}, lambda={s.lam} A, l_osv={L_OSV}), A0 only",
                      "osv_method": args.osv_method, "osv_prec": args.prec, "b_mode": "regen",
                      "n_osv_min": int(n_osv.min()), "n_osv_max": int(n_osv.max()),
                      "n_osv_mean": float(np.mean(n_osv)),
                      "l2": "256 MB buffer written between timed steps"},
           "gpu_launches": int(pkg.osvmp2.kernel_launches() - launches0),
           "phases": {k: {"ms_per_step": v[0] / args.steps,
                          "tflops": (v[1] / (v[0] / 1e3) / 1e12) if v[0] > 0 and v[1] else None}
                      for k, v in prof.items()},
           "clocks": clk.summary()}
    if not args.no_cpu_baseline:
        import oracle
        chk = {}
        for i in (0, s.n_occ // 2):
            Qg, wg = (x.cpu().numpy() for x in ctx.get_osv(i))
            T = oracle.semicanonical_tii(s.B_block(i), s.e_vir, s.f_occ[i, i])
            if args.osv_method == "randomized":
                ro = oracle.randomized_osv(T, L_OSV, lambda k, i=i: synth.gauss_row(s.seed, i, k, s.n_vir))
                Qr, wr = ro.Q, ro.omega
            else:
                Qr, wr = oracle.osv_from_tii(T, L_OSV)
            same = Qg.shape[1] == Qr.shape[1]
            chk[str(i)] = {"n_osv": int(Qg.shape[1]), "n_osv_oracle": int(Qr.shape[1]),
                           "omega_max_rel_err": float(np.abs(wg - wr).max() / wr.max()) if same else None,
                           "projector_max_err": float(np.abs(Qg @ Qg.T - Qr @ Qr.T).max()) if same else None}
        out["osv_vs_oracle"] = chk
    print(json.dumps(out), flush=True)
    ctx.close()


def gradient_vs_oracle(s, dB0, osv_method="exact", relaxed=False):
    """dE/dB[0] from the oracle, summed over the fragments that contain orbital 0,
    against the GPU's row block (same OSV rule); with relaxed, plus the response of
    Q_0 to T_00, which only those fragments feed."""
    import oracle
    frags = [(o, c) for o, c in oracle.mbe3_fragments(s.r_occ, R2_CUT, R3_CUT) if 0 in o and c != 0]
    orbs = sorted({x for o, _ in frags for x in o})
    t0 = time.perf_counter()
    osys = oracle.OSVSystem(s.B_block, s.n_occ, s.e_vir, s.f_occ, l_osv=L_OSV, orbitals=orbs)
    ref = np.zeros((s.n_vir, s.n_aux))
    G0 = 0.0
    for o, c in frags:
        fr = osys.fragment(o)
        res = oracle.solve_fragment(fr)
        gB, _, _ = oracle.fragment_gradient(fr, res, osys.B, s.n_occ, s.n_vir, s.n_aux)
        ref += c * gB[0]
        if relaxed:
            G0 = G0 + c * oracle.fragment_dE_dQ(fr, res, osys.B, s.e_vir)[0]
    if relaxed:
        T00 = oracle.semicanonical_tii(osys.B(0), s.e_vir, s.f_occ[0, 0])
        Z, _ = oracle.osv_response(T00, osys.Q[0], G0)
        ref += oracle.tii_adjoint(Z, osys.B(0), s.e_vir, s.f_occ[0, 0])[0]
    err = float(np.abs(dB0 - ref).max())
    return {"rows": "dE/dB[0] (every fragment containing orbital 0)" + (", OSVs relaxed" if relaxed else ""),
            "fragments": len(frags),
            "max_abs": err, "max_rel": err / float(np.abs(ref).max()), "oracle_s": time.perf_counter() - t0}


def cpu_baseline(args, budget_s: float):
    done, dt, k, energies = cpu_sample(args, budget_s)
    return ({"value": done / dt, "unit": "fragments/s", "cores": os.cpu_count(), "kind": "oracle",
             "sample": f"OSV build of the {k} orbitals nearest orbital 0 + the {done} MBE(3) fragments inside "
                       f"that set ({dt:.1f} s, NumPy FP64, BLAS threads = all cores)"}, energies)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    for _ in range(args.warmup):
        cpu_sample(args, args.cpu_budget)
    vals, times, frags = [], [], 0
    for _ in range(args.steps):
        done, dt, k, _ = cpu_sample(args, args.cpu_budget)
        vals.append(done / dt)
        times.append(dt)
        frags = done
    v = statistics.median(vals)
    print(json.dumps({
        "impl": "reference", "metric": "MBE(3) fragments/s", "value": v, "unit": "fragments/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.workload} (bounded sample, {args.cpu_orbitals} orbitals)"},
        "cpu_baseline": {"value": v, "unit": "fragments/s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": f"{frags} fragments among the {args.cpu_orbitals} orbitals nearest orbital 0"},
        "e2e": {"value": v, "unit": "fragments/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--prec", choices=["fp64", "mixed"], default="mixed")
    ap.add_argument("--workload", default="mbe3_n128", choices=sorted(synth.WORKLOADS))
    ap.add_argument("--b-mode", choices=["regen", "stored"], default="regen")
    ap.add_argument("--grad", action="store_true")
    ap.add_argument("--relaxed", action="store_true",
                    help="with --grad: the OSV-relaxed gradient (FP64 form, exact OSVs)")
    ap.add_argument("--osv-method", choices=["exact", "randomized"], default="exact",
                    help="OSV generation: full eigen-decomposition or the randomized range finder (Algorithm 3)")
    ap.add_argument("--osv-only", action="store_true",
                    help="time the OSV build (A0) alone, in orbitals/s")
    ap.add_argument("--screen", action="store_true",
                    help="cluster selection by s2b/s3b with weak pairs instead of the 8/6 A distance rule")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--cpu-budget", type=float, default=25.0)
    # 16 orbitals: 293 fragments, 18.3 per OSV build (the full workload has 23.8)
    ap.add_argument("--cpu-orbitals", type=int, default=16)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--measure-peaks", action="store_true",
                    help="print the FP64 / TF32 / FP32 / BF16 GEMM throughput of GPU 0 and exit")
    args = ap.parse_args()
    if args.relaxed and not (args.grad and args.prec == "fp64" and args.osv_method == "exact"):
        ap.error("--relaxed needs --grad --prec fp64 with exact OSVs")
    if args.measure_peaks:
        print(json.dumps(measure_peaks()), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
