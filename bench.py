#!/usr/bin/env python
"""Throughput of one semi-implicit CH / AC / NS step on GB300.

Workload (default): the 1024 x 1024 structured thin-film mesh (1,050,625 P1
nodes, 4,198,401 P2 velocity nodes), eps = 0.005, dt = 5e-4, FP32
multigrid / Chebyshev preconditioners inside FP64 FGMRES at a 1e-8 relative
residual.  Inputs are synthetic (seeded SplitMix64 noise on the polymer and
NFA fractions); the per-step working set (> 10 GB) is far larger than L2.

A timed step = assembly + 3 Cahn-Hilliard solves + Allen-Cahn + air
potential + Navier-Stokes (chnss_step on device buffers); the trajectory
advances from step to step.  One JSON line on rank 0.

  python bench.py [--steps K] [--warmup W] [--gpus N]
  python bench.py --impl reference     # the CPU oracle on the same metric
  python bench.py --sweep              # 64 independent instances, chnss_step_batched
  python bench.py --adjoint            # gradient through 40 FP64 steps on 256 x 256
  python bench.py --amg                # smoothed-aggregation AMG on the CH block M + tau C(v)
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "film1024_mixed"
CPU_SAMPLE_N = 256          # cpu_baseline: one oracle step on 256 x 256 (~10-30 s)
REF_SAMPLE_N = 128          # --impl reference: one oracle step on 128 x 128 per timed step
METRIC = "time steps/s at 1M nodes (1024x1024 P1 mesh, FGMRES to 1e-8 relative residual)"
FP64_FMA_PER_SM_CLK = 2     # FP64 FMA issue rate per multiprocessor per clock on this part


# GB300 HBM3e nominal bandwidth (8 stacks), reported beside the measured copy
# bandwidth that the fractions are taken against
HBM_NOMINAL_GBS = 7900.0


def fp64_peak_tflops(sm_max_mhz=None):
    """ALU roof of FP64 work: multiprocessors of the current device x FP64
    FMAs per clock x 2 FLOP x the maximum SM clock (sampled by nvidia-smi
    during the run, else the measured one, else 2070 MHz)."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = sm_max_mhz
    if not mhz:
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                mhz = float(json.load(f)["sm_max_mhz"])
        except Exception:
            mhz = 2070.0
    return sms * FP64_FMA_PER_SM_CLK * 2 * mhz * 1e6 / 1e12, sms, mhz


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def nodes(n):
    return (n + 1) ** 2


# ---------------------------------------------------------------------------
def cpu_sample(n: int, workload: str, steps: int = 1) -> dict:
    """One oracle step (plain numpy/scipy, FP64) of the workload's parameter
    set on an n x n mesh; returns seconds per step."""
    from oracle.step import Oracle
    from paper_2501_11767_gb300 import inputs
    w = inputs.workload(workload)
    params = dict(w["params"], precision=0)
    o = Oracle(n, params)
    init = inputs.initial_state_solvent_air if w.get("init") == "solvent_air" else inputs.initial_state
    st = init(n, seed=0)
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        st, info = o.step(st)
        times.append(time.perf_counter() - t0)
    return {"n": n, "seconds": times, "iters": {k: v["iters"] for k, v in info.items() if isinstance(v, dict)}}


def run_cpu_sample_subprocess(n: int, workload: str, steps: int = 1) -> dict:
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample", str(n), "--cpu-steps", str(steps),
                        "--workload", workload], capture_output=True, text=True, env=env, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id=None):
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"chnss_clocks_{os.getpid()}_{id(self)}.csv")
        self.device_id = device_id

    def start(self):
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.device_id:
                cmd[1:1] = ["-i", self.device_id]
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2501_11767_gb300 import chnss, inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    def barrier():
        if world > 1:
            dist.barrier()

    w = inputs.workload(args.workload)
    n, params = w["n"], dict(w["params"])
    if args.ortho >= 0:
        params["ortho"] = args.ortho
    mesh = chnss.Mesh(n, top_bc=params.get("top_bc", 0))
    N1, N2 = mesh.N1, mesh.N2
    stream = torch.cuda.current_stream()
    init = inputs.initial_state_solvent_air if w.get("init") == "solvent_air" else inputs.initial_state
    st0 = chnss.state_to_device(init(n, seed=rank))

    def timed_run(prm, warmup, steps, profile, concurrent=True):
        ctx = chnss.Context(mesh, prm, stream)
        ctx.set_step_concurrency(concurrent)
        if args.step_mode == 1 and not profile:
            ctx.set_step_mode(1)
        a, b = {k: v.clone() for k, v in st0.items()}, ctx.new_state()
        for _ in range(warmup):
            ctx.step(a, b)
            a, b = b, a
        torch.cuda.synchronize()
        diag0 = ctx.diagnostics(a)             # outside the timed region
        ctx.profile_enable(profile)
        launches0 = ctx.profile_read()["launches"]
        sampler = ClockSampler(_device_uuid(torch, local))
        barrier()
        torch.cuda.synchronize()
        sampler.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        infos = []
        e0.record(stream)
        for _ in range(steps):
            _, info, status = ctx.step(a, b)
            infos.append(info)
            a, b = b, a
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        clocks = sampler.stop()
        ms = e0.elapsed_time(e1)
        prof = ctx.profile_read()
        ctx.profile_enable(False)
        timed_run.launches_before = launches0
        timed_run.last_state = a
        timed_run.diag = (diag0, ctx.diagnostics(a))
        return ctx, ms, infos, prof, prof["launches"] - launches0, clocks

    # headline: the library's default step (CH, AC and NS solved concurrently), no probes
    ctx, ms, infos, _, launches, clocks = timed_run(params, args.warmup, args.steps, False)
    launches_before_timed = timed_run.launches_before
    state_after = timed_run.last_state
    conservation = conservation_record(*timed_run.diag, args.steps, params)
    inner = None
    if params.get("inner_rtol", 0.0) > 0:
        inner = {"inner_rtol": params["inner_rtol"], "inner_maxit": params["inner_maxit"],
                 "over": "warm-up and timed steps",
                 "blocks": {b: {"solves": v["solves"], "vcycles_per_solve": round(v["cycles"] / v["solves"], 2)}
                            for b, v in ctx.inner_stats().items() if v["solves"]},
                 "gpu_launches_note": "a WHILE-node body counts once per graph launch, not once per V-cycle"}
    ms_t = torch.tensor([ms], device=dev)
    if world > 1:
        dist.all_reduce(ms_t, op=dist.ReduceOp.MAX)
    ms_max = float(ms_t.item())
    value = world * args.steps / (ms_max / 1e3)

    # end to end through the C ABI with host buffers (pinned), copies inside
    e2e = None
    if not args.no_e2e:
        host_in = {k: torch.empty(v.shape, dtype=torch.float64, pin_memory=True).numpy() for k, v in st0.items()}
        host_out = {k: torch.empty(v.shape, dtype=torch.float64, pin_memory=True).numpy() for k, v in st0.items()}
        # continue the trajectory of the timed region (same iteration regime)
        for k, v in state_after.items():
            host_in[k][...] = v.cpu().numpy()
        ctx.step_host(host_in, host_out)            # warm-up (allocates the staging buffers)
        host_in, host_out = host_out, host_in
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        e2e_infos = []
        for _ in range(args.e2e_steps):
            _, inf_h, _ = ctx.step_host(host_in, host_out)
            e2e_infos.append(inf_h)
            host_in, host_out = host_out, host_in
        t_e2e = time.perf_counter() - t0
        t_t = torch.tensor([t_e2e], device=dev)
        if world > 1:
            dist.all_reduce(t_t, op=dist.ReduceOp.MAX)
        nbytes = (9 * N1 + 2 * N2) * 8
        e2e = {"value": world * args.e2e_steps / float(t_t.item()), "unit": "steps/s",
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "steps": args.e2e_steps,
               "iters_mean": {k: round(sum(i[k]["iters"] for i in e2e_infos) / len(e2e_infos), 2) for k in e2e_infos[0]},
               "trajectory": "continues from the state after the timed region",
               "how": "chnss_step_host: pinned host state in, H2D copy, step, D2H copy, stream sync; wall clock"}
    del ctx

    # roofline region: the same workload with every solve alone on the stream
    # (serial step) and CUDA-event probes around the instrumented kernels, so
    # that each family's duration is not shared with concurrent solves
    ms_r, prof = 0.0, {"kinds": {}}
    if args.roofline_steps > 0:
        ctxr, ms_r, _, prof, _, _ = timed_run(params, args.warmup, args.roofline_steps, True, concurrent=False)
        del ctxr

    bf16 = None
    if args.bf16_steps > 0:
        pb = dict(params, precision=2)
        ctxb, msb, infosb, _, _, _ = timed_run(pb, args.warmup, args.bf16_steps, False)
        del ctxb
        bf16 = {"value": args.bf16_steps / (msb / 1e3), "unit": "steps/s", "steps": args.bf16_steps,
                "ms_per_step": msb / args.bf16_steps,
                "what": "precision 2: velocity multigrid values stored in BF16, FP32 vectors, FP64 FGMRES",
                "converged": all(i[k]["converged"] for i in infosb for k in i),
                "iters_mean": {k: round(sum(i[k]["iters"] for i in infosb) / len(infosb), 2) for k in infosb[-1]},
                "iters_last_step": {k: v["iters"] for k, v in infosb[-1].items()}}

    fp64 = None
    if not args.no_fp64 and args.fp64_steps > 0:
        p64 = dict(params, precision=0, ortho=0)     # FP64 throughout, Gram-Schmidt included
        ctx64, ms64, infos64, _, _, _ = timed_run(p64, 1, args.fp64_steps, False)
        fp64 = {"value": args.fp64_steps / (ms64 / 1e3), "unit": "steps/s", "steps": args.fp64_steps,
                "ms_per_step": ms64 / args.fp64_steps,
                "iters_last_step": {k: v["iters"] for k, v in infos64[-1].items()}}
        # error of the mixed-precision step against the FP64 step, both from
        # the state after the headline timed region (one step each)
        mixed_vs_fp64 = None
        if params["precision"] != 0:
            out64, i64, _ = ctx64.step(state_after)
            got64 = chnss.state_to_numpy(out64)
            del ctx64, out64
            ctxm = chnss.Context(mesh, params, stream)
            outm, im, _ = ctxm.step(state_after)
            gotm = chnss.state_to_numpy(outm)
            del ctxm, outm
            rel = lambda a, b: float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))  # noqa: E731
            mixed_vs_fp64 = {
                "rel_l2": {"phi": rel(gotm["phi"], got64["phi"]), "mu": rel(gotm["mu"], got64["mu"]),
                           "Phi_v": rel(gotm["Phi_v"], got64["Phi_v"]), "v": rel(gotm["v"], got64["v"]),
                           "p": rel(gotm["p"], got64["p"])},
                "iters": {"mixed": {k: v["iters"] for k, v in im.items()},
                          "fp64": {k: v["iters"] for k, v in i64.items()}},
                "how": "one step of each precision from the same state (the state after the timed region), "
                       f"both to a {params['rtol']:g} relative residual; relative L2 of mixed - FP64 per field "
                       "(the FP64 path is checked against the oracle at 1e-9 per solve on the smaller meshes)"}
        else:
            del ctx64
        fp64["mixed_vs_fp64"] = mixed_vs_fp64

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # roofline of the dominant kernel family (largest summed event time);
    # FP64 families that need more than one FMA per 11 bytes are bound by the
    # FP64 pipe of this part, not by HBM
    peak, peak_kind = peaks()
    fp64_peak, n_sms, peak_mhz = fp64_peak_tflops(clocks["sm_max_mhz"] if clocks else None)
    kinds = {k: v for k, v in prof["kinds"].items() if v["launches"] > 0 and v["bytes"] > 0}

    def family_roofline(name):
        d = kinds[name]
        ms_l = d["ms"] / d["launches"]
        gbps = d["bytes"] / (d["ms"] * 1e-3) / 1e9
        # FP64 balance point, FLOP per byte of the measured HBM bandwidth (~0.19)
        if d.get("flops", 0.0) > 0 and d["flops"] / d["bytes"] > fp64_peak * 1e12 / (peak * 1e9):
            tf = d["flops"] / (d["ms"] * 1e-3) / 1e12
            return {"kernel": name, "bound": "alu", "achieved": round(tf, 4), "peak": round(fp64_peak, 4),
                    "unit": "TFLOP/s", "frac": round(tf / fp64_peak, 4),
                    "peak_source": f"derived: {n_sms} SMs x {FP64_FMA_PER_SM_CLK} FP64 FMA/clk x 2 FLOP x "
                                   f"{peak_mhz:.0f} MHz",
                    "flops_per_launch": d["flops"] / d["launches"], "bytes_per_launch": d["bytes"] / d["launches"],
                    "ms_per_launch": ms_l, "launches": d["launches"], "hbm_GBps": round(gbps, 1),
                    "hbm_frac": round(gbps / peak, 4), "traffic": _traffic(name, d["bytes"] / d["launches"])}
        return {"kernel": name, "bound": "hbm", "achieved": round(gbps, 1), "peak": peak, "unit": "GB/s",
                "frac": round(gbps / peak, 4), "peak_source": peak_kind,
                "frac_of_nominal": round(gbps / HBM_NOMINAL_GBS, 4),
                "bytes_per_launch": d["bytes"] / d["launches"], "ms_per_launch": ms_l,
                "launches": d["launches"], "traffic": _traffic(name, d["bytes"] / d["launches"])}

    roofline = family_roofline(max(kinds, key=lambda k: kinds[k]["ms"])) if kinds else None
    rooflines = {k: family_roofline(k) for k in kinds}
    families = {k: {"ms_total": round(v["ms"], 3), "launches": v["launches"],
                    "GBps": round(v["bytes"] / (v["ms"] * 1e-3) / 1e9, 1) if v["ms"] > 0 and v["bytes"] > 0 else None,
                    "share_of_step": round(v["ms"] / ms_r, 4)}
                for k, v in prof["kinds"].items() if v["launches"] > 0}

    cpu = None
    if not args.no_cpu and world == 1:
        try:
            smp = run_cpu_sample_subprocess(CPU_SAMPLE_N, args.workload)
            sec = smp["seconds"][0]
            cpu = {"value": (1.0 / sec) * nodes(CPU_SAMPLE_N) / nodes(n), "unit": "steps/s", "cores": 1,
                   "kind": "oracle", "calibration": oracle_calibration(),
                   "sample": f"one oracle step (numpy/scipy FP64, 1 thread) of the same parameter set on a "
                             f"{CPU_SAMPLE_N}x{CPU_SAMPLE_N} mesh ({nodes(CPU_SAMPLE_N)} nodes) in {sec:.1f} s, "
                             f"scaled by the node ratio to the {n}x{n} mesh",
                   "cpu": cpu_model(), "host_cores": os.cpu_count(), "iters": smp["iters"]}
        except Exception as e:  # reported, not fatal
            cpu = {"value": None, "error": str(e)[-300:]}

    last = infos[-1]
    out = {
        "metric": workload_metric(args.workload, n, params), "value": round(value, 4), "unit": "steps/s",
        "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64 outer / f32 preconditioner",
        "data": "synthetic (seeded SplitMix64 noise on phi_p, phi_NFA; paper-shaped thin film)",
        "config": {"workload": args.workload, "n": n, "p1_nodes": N1, "p2_nodes": N2,
                   "velocity_dofs": 2 * N2, "precision": "mixed" if params["precision"] == 1 else "fp64",
                   "gram_schmidt": "double-FP32" if params.get("ortho", 0) == 1 else "FP64",
                   "step_mode": "one graph" if args.step_mode == 1 else "host-driven Krylov loops",
                   "rtol": params["rtol"], "restart": params["restart"], "tau": params["tau"],
                   "beta": params["beta"],
                   "l2": "inputs larger than L2 (per-step working set > 10 GB)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "iters_last_step": {k: v["iters"] for k, v in last.items()},
        "solve_seconds_last_step": {k: round(v["seconds"], 4) for k, v in last.items()},
        "iters_mean": {k: round(sum(i[k]["iters"] for i in infos) / len(infos), 2) for k in last},
        "converged": all(i[k]["converged"] for i in infos for k in last),
        "fp64": fp64,
        "speedup_mixed_vs_fp64": round(value / fp64["value"], 3) if fp64 else None,
        "bf16_preconditioner": bf16,
        "inner_multigrid": inner,
        "conservation": conservation,
        "roofline": roofline,
        "roofline_region": {"steps": args.roofline_steps, "warmup": args.warmup,
                            "ms_per_step": round(ms_r / args.roofline_steps, 3) if args.roofline_steps else None,
                            "how": "separate timed region, solves one after the other (chnss_set_step_concurrency 0), "
                                   "CUDA events around each instrumented launch on its stream; the headline value "
                                   "comes from the concurrent region without probes"},
        "rooflines": rooflines,
        "kernel_families": families,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "gpu_launches_before_timed": launches_before_timed,
        "clocks": clocks,
    }
    print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def conservation_record(d0, d1, steps, params):
    """Mass, divergence and energy of the trajectory over the timed steps
    (chnss_diagnostics: FP64 deterministic sums on the device)."""
    drift = [abs(d1["mass"][i] - d0["mass"][i]) / max(abs(d0["mass"][i]), 1e-300) for i in range(3)]
    return {"steps": steps,
            "mass_rel_drift": {"phi_p": drift[0], "phi_N": drift[1], "phi_s": drift[2]},
            "mass_before": d0["mass"], "mass_after": d1["mass"],
            "div_norm_after": d1["div"], "p_mean_after": d1["p_mean"],
            "energy_before": d0["energy"], "energy_after": d1["energy"],
            "enclosed": params.get("top_bc", 0) == 0,
            "how": "chnss_diagnostics before and after the timed steps (outside the timed region); for enclosed "
                   "flow the scheme conserves int phi_i exactly, so the drift is the solves' residual level"}


def _device_uuid(torch, idx):
    try:
        u = str(torch.cuda.get_device_properties(idx).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


def _traffic(kernel, bytes_per_launch):
    """DRAM bytes per launch of a family from the committed ncu summary
    (profiles/traffic.json): the measured DRAM / algorithmic byte ratio of
    the family's kernels on a smaller capture, times this launch's
    algorithmic bytes (traffic grows with the vectors swept)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        ratio = d[kernel]["dram_per_algorithmic_byte"]
        return round(ratio * bytes_per_launch)
    except Exception:
        return None


# ---------------------------------------------------------------------------
def workload_metric(name, n, params):
    """The headline metric for the headline workload; other workloads name
    their own mesh and stopping rules."""
    if name == WORKLOAD:
        return METRIC
    rule = f"FGMRES to {params['rtol']:g} relative residual"
    if params.get("ns_rtol", 0.0) > 0:
        rule += f" (Oseen {params['ns_rtol']:g}, absolute {params['atol']:g} / {params['ns_atol']:g})"
    if params.get("inner_rtol", 0.0) > 0:
        rule += f", inner multigrid to {params['inner_rtol']:g}"
    return f"time steps/s, {name} ({n}x{n} P1 mesh, {rule})"


SWEEP_METRIC = "aggregate time steps/s of a 64-instance parameter sweep (meshes 128^2..512^2, FGMRES to 1e-8)"


def shard(items: list, rank: int, world: int) -> list:
    """Instances of one rank: round-robin over the sweep (independent
    problems, no data-path collective)."""
    return [x for i, x in enumerate(items) if i % world == rank]


ADJOINT_METRIC = "gradients/s of J = int |grad phi_p(t_40)|^2 on 256x256 (40 FP64 steps, checkpoints every 8)"


def run_adjoint(args):
    """The adjoint workload: one full gradient of the final-morphology
    functional with respect to (evaporation rate, mobility scale, initial
    polymer field) through 40 FP64 steps on 256 x 256, with a checkpoint
    every 8 steps (forward sweep, segment recomputation, adjoint steps);
    with --three-d, 20 FP64 3D steps on the Kuhn mesh of --three-d-n cubes,
    checkpoints every 4.  A timed unit is one whole gradient."""
    import torch

    from paper_2501_11767_gb300 import adjoint, chnss, inputs

    torch.cuda.set_device(0)
    if args.three_d:   # the 3D adjoint (chnss3_adjoint_step) on the Kuhn mesh of n^3 cubes
        n, steps, every = args.three_d_n, 20, 4
        p = dict(inputs.default_params(), tau=1e-4, mobility_kind=1)
        ctx = chnss.Context3(n, p)
        st0 = chnss.state_to_device(inputs.initial_state_3d(n, seed=0))
        workload = f"adjoint3d{n}"
    else:
        n, steps, every = 256, 40, 8
        p = inputs.workload("film256_mobility")["params"]   # concentration-dependent mobility
        ctx = chnss.Context(chnss.Mesh(n), p)
        st0 = chnss.state_to_device(inputs.initial_state(n, seed=0))
        workload = "adjoint256"
    for _ in range(args.warmup):
        adjoint.trajectory_gradient(ctx, st0, 2, checkpoint_every=1)
    torch.cuda.synchronize()
    sampler = ClockSampler(_device_uuid(torch, 0))
    sampler.start()
    t0 = time.perf_counter()
    g = None
    for _ in range(args.steps):
        g = adjoint.trajectory_gradient(ctx, st0, steps, checkpoint_every=every)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    clocks = sampler.stop()
    # forward steps per gradient: the sweep plus the recomputed segments
    fwd = steps + sum(min(every, steps - k) for k in range(0, steps, every))
    out = {
        "metric": ADJOINT3_METRIC.format(n=n) if args.three_d else ADJOINT_METRIC,
        "value": round(args.steps / sec, 4), "unit": "gradients/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(sec / args.steps * 1e3, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded SplitMix64 noise on phi_p, phi_NFA)",
        "config": {"workload": workload, "n": n, "time_steps": steps, "checkpoint_every": every,
                   "forward_steps_per_gradient": fwd, "adjoint_steps_per_gradient": steps,
                   "adjoint_rtol": 1e-12, "forward_rtol": p["rtol"], "beta": p["beta"],
                   "mobility": "gamma (phi (1 - phi) + m0)" if p["mobility_kind"] else "constant"},
        "J": g["J"], "dJ_devap": g["evap"], "dJ_dgamma": g["gamma"],
        "timing": "wall clock around trajectory_gradient (forward sweep, checkpoints, recomputation, adjoint steps)",
        "clocks": clocks,
    }
    print(json.dumps(out))


ADJOINT3_METRIC = ("gradients/s of J = int |grad phi_p|^2 after 20 FP64 3D steps on the Kuhn mesh of {n}^3 "
                   "cubes (discrete adjoint, checkpoints every 4)")
THREE_D_METRIC = ("time steps/s of the 3D step on the Kuhn mesh of {n}^3 cubes "
                  "(FP32 multigrid inside FP64 FGMRES to 1e-8)")


def run_three_d(args):
    """The 3D workload (the paper's 3D runs, Sec. 5, on a Kuhn tetrahedral
    mesh): the film parameter set with the 3D step (chnss3_step): FP32
    multigrid inside FP64 FGMRES with double-FP32 Gram-Schmidt (the
    headline), the same with BF16 velocity values, and FP64 throughout; the
    three solve groups concurrent on their streams; CUDA events around the
    timed steps, inputs resident on the device."""
    import torch

    from paper_2501_11767_gb300 import chnss, inputs

    torch.cuda.set_device(0)
    n = args.three_d_n
    p = inputs.default_params()
    p.update(tau=1e-4)                 # the 3D figures' time step (Sec. 5)
    if args.three_d_mobility:          # gamma_i (phi_i (1 - phi_i) + m0), lagged
        p.update(mobility_kind=1)
    if args.three_d_open:              # do-nothing top face
        p.update(top_bc=1)
    if args.three_d_inner > 0:         # multigrid blocks iterated to a tolerance (Sec. 5: 1e-4)
        p.update(inner_rtol=args.three_d_inner, inner_maxit=20)
    stream = torch.cuda.current_stream()

    if args.nvtx_step:
        # one serial mixed step inside the NVTX range "step" (for an ncu launch
        # list: --nvtx --nvtx-include "step/"), after the warm-up steps
        ctx = chnss.Context3(n, dict(p, precision=1, ortho=1), stream)
        ctx.set_step_concurrency(False)
        a = chnss.state_to_device(inputs.initial_state_3d(n, seed=0))
        b = ctx.new_state()
        for _ in range(args.warmup):
            ctx.step(a, b)
            a, b = b, a
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("step")
        _, info, _ = ctx.step(a, b)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"nvtx_step": f"film3d{n}_mixed", "iters": {k: v["iters"] for k, v in info.items()}}))
        return

    def timed(prm):
        ctx = chnss.Context3(n, prm, stream)
        a = chnss.state_to_device(inputs.initial_state_3d(n, seed=0))
        b = ctx.new_state()
        for _ in range(args.warmup):
            ctx.step(a, b)
            a, b = b, a
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        infos = []
        e0.record(stream)
        for _ in range(args.steps):
            _, info, _ = ctx.step(a, b)
            infos.append(info)
            a, b = b, a
        e1.record(stream)
        torch.cuda.synchronize()
        return ctx, e0.elapsed_time(e1), infos

    sampler = ClockSampler(_device_uuid(torch, 0))
    sampler.start()
    ctx, ms, infos = timed(dict(p, precision=1, ortho=1))
    clocks = sampler.stop()
    _, ms64, infos64 = timed(dict(p, precision=0))
    _, ms16, infos16 = timed(dict(p, precision=2, ortho=1))
    iters = lambda inf: {k: round(sum(i[k]["iters"] for i in inf) / len(inf), 2) for k in inf[-1]}   # noqa: E731
    value = args.steps / (ms / 1e3)
    fp64 = args.steps / (ms64 / 1e3)
    out = {
        "metric": THREE_D_METRIC.format(n=n), "value": round(value, 4), "unit": "steps/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64 outer / f32 preconditioner",
        "data": "synthetic (seeded SplitMix64 noise on phi_p, phi_NFA)",
        "config": {"workload": f"film3d{n}{'_mobility' if args.three_d_mobility else ''}"
                               f"{'_open' if args.three_d_open else ''}{'_inner' if args.three_d_inner > 0 else ''}_mixed",
                   "n": n, "mobility": "phi (1 - phi) + m0" if args.three_d_mobility else "constant",
                   "top": "open (do-nothing)" if args.three_d_open else "no-slip",
                   "inner_rtol": args.three_d_inner, "p1_nodes": ctx.N1, "p2_nodes": ctx.N2,
                   "velocity_dofs": 3 * ctx.N2, "tau": p["tau"], "rtol": p["rtol"], "parallelism": "single GPU",
                   "l2": "inputs larger than L2" if 3 * ctx.N2 * 8 * 100 > 129e6 else "working set near L2"},
        "iters_mean": iters(infos),
        "converged": all(i[k]["converged"] for i in infos for k in i),
        "fp64": {"value": round(fp64, 4), "unit": "steps/s", "ms_per_step": round(ms64 / args.steps, 2),
                 "iters_mean": iters(infos64)},
        "bf16_velocity": {"value": round(args.steps / (ms16 / 1e3), 4), "unit": "steps/s",
                          "ms_per_step": round(ms16 / args.steps, 2), "iters_mean": iters(infos16),
                          "converged": all(i[k]["converged"] for i in infos16 for k in i)},
        "speedup_mixed_vs_fp64": round(value / fp64, 3),
        "clocks": clocks,
    }
    print(json.dumps(out))


AMG_METRIC = ("SA-AMG re-setups + solves/s of the Cahn-Hilliard block M + tau C(v) at {n}x{n} "
              "(numeric setup on the step's new values, then SA-preconditioned FGMRES to 1e-8)")


def run_amg(args):
    """The paper's per-step use of smoothed aggregation (Sec. 5: SA for the
    nonsymmetric Cahn-Hilliard blocks): the block L = M + tau C(v) of the
    1024^2 film workload, assembled by the library after args.warmup mixed
    steps (so that C(v) carries the flow), is given to chnss_amg_create
    (symbolic + numeric setup, timed once); a timed repetition is
    chnss_amg_update on the current values (spectral bounds, prolongators,
    Galerkin products, smoother data) followed by chnss_amg_solve of L x = b
    (b: the polymer CH right-hand side's first block) in FP64 and FP32
    hierarchies.  CUDA events on the handle's synchronised calls, inputs
    resident on the device."""
    import numpy as np
    import torch

    from paper_2501_11767_gb300 import chnss, inputs

    torch.cuda.set_device(0)
    w = inputs.workload(args.workload)
    n, params = w["n"], dict(w["params"])
    mesh = chnss.Mesh(n)
    stream = torch.cuda.current_stream()
    ctx = chnss.Context(mesh, params, stream)
    a, b = chnss.state_to_device(inputs.initial_state(n, seed=0)), ctx.new_state()
    for _ in range(args.warmup):
        ctx.step(a, b)
        a, b = b, a
    ctx.assemble(a)
    rp, col, val = ctx.export_csr(0)
    rhs = ctx.export_rhs(0)[:mesh.N1]
    torch.cuda.synchronize()
    d = lambda x, t: torch.as_tensor(x, dtype=t, device="cuda")   # noqa: E731
    rp_d, col_d, val_d, b_d = d(rp, torch.int32), d(col, torch.int32), d(val, torch.float64), d(rhs, torch.float64)
    out = {}
    sampler = ClockSampler(_device_uuid(torch, 0))
    for prec, key in ((1, "fp32_hierarchy"), (0, "fp64_hierarchy")):
        t0 = time.perf_counter()
        h = chnss.Amg(rp_d, col_d, val_d, precision=prec)
        create_s = time.perf_counter() - t0
        for _ in range(2):                        # warm-up repetitions
            h.update(val_d)
            h.solve(b_d, rtol=1e-8)
        torch.cuda.synchronize()
        if prec == 1:
            sampler.start()
            torch.cuda.nvtx.range_push("amg")      # the timed FP32-hierarchy repetitions (ncu --nvtx-include)
        t_upd, t_sol, iters = [], [], []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            h.update(val_d)
            t1 = time.perf_counter()
            x, info, _ = h.solve(b_d, rtol=1e-8)
            t2 = time.perf_counter()
            t_upd.append(t1 - t0)
            t_sol.append(t2 - t1)
            iters.append(info["iters"])
        if prec == 1:
            torch.cuda.nvtx.range_pop()
            clocks = sampler.stop()
        xr = x.cpu().numpy()
        Lx = np.zeros(mesh.N1)
        np.add.at(Lx, np.repeat(np.arange(mesh.N1), np.diff(rp)), val * xr[col])
        res = float(np.linalg.norm(rhs - Lx) / np.linalg.norm(rhs))
        out[key] = {"create_s": round(create_s, 3), "update_ms": round(1e3 * statistics.median(t_upd), 2),
                    "solve_ms": round(1e3 * statistics.median(t_sol), 2), "iters": iters[-1],
                    "rel_residual": res, "levels": h.levels(),
                    "value": round(args.steps / (sum(t_upd) + sum(t_sol)), 3)}
        h.close()
    head = out["fp32_hierarchy"]
    line = {
        "metric": AMG_METRIC.format(n=n), "value": head["value"], "unit": "setups+solves/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(head["update_ms"] + head["solve_ms"], 2), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64 outer / f32 hierarchy",
        "data": f"synthetic (the {n}^2 film state after the warm-up steps)",
        "config": {"workload": f"amg_ch_block{n}", "n": n, "rows": mesh.N1, "nnz": int(len(col)),
                   "tau": params["tau"], "rtol": 1e-8, "parallelism": "single GPU",
                   "l2": ("matrices of the hierarchy larger than L2" if 12 * len(col) * 2 > 129e6
                          else "hierarchy near the L2 size (a profiling size)")},
        "clocks": clocks, **out,
    }
    print(json.dumps(line))


def run_sweep(args):
    """Batched parameter sweep (the 64-instance workload): independent
    instances of uneven mesh size and evaporation rate, one context (and
    stream) each, FP32 preconditioners inside FP64 FGMRES with double-FP32
    Gram-Schmidt.  Headline: every instance step one recorded CUDA graph
    (chnss_set_step_mode 1), all instances launched by chnss_step_batched
    from one thread, args.sweep_steps steps each; beside it the whole batch
    as one graph launch per batch step (chnss_set_batch_mode 1).  Beside it: the same batch
    host-driven (worker threads, one synchronisation per Krylov iteration),
    and the instances' FP64 steps one instance at a time.  Under torchrun the
    instances are sharded round-robin over the ranks (a fixed sweep: strong
    scaling)."""
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2501_11767_gb300 import chnss, inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if world > 1:
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            dist.barrier()

    all_inst = inputs.sweep_instances(args.sweep_count)
    inst = shard(all_inst, rank, world)
    meshes = {n: chnss.Mesh(n) for n in sorted({i["n"] for i in inst})}
    tuning = {}
    for n, m in meshes.items():          # tune each mesh on a throw-away context
        c = chnss.Context(m, inst[0]["params"])
        c.step(chnss.state_to_device(inputs.initial_state(n, seed=0)))
        tuning[n] = c.autotune()
        del c
    threads = args.sweep_threads or min(16, os.cpu_count() or 1)

    def make(mode, params_of=lambda i: i["params"]):
        ctxs = [chnss.Context(meshes[i["n"]], params_of(i), stream=torch.cuda.Stream()) for i in inst]
        for c in ctxs:
            c.set_step_mode(mode)
            if mode == 0 and not args.sweep_concurrent_steps:
                c.set_step_concurrency(False)   # host-driven: the instances overlap already
        a = [chnss.state_to_device(inputs.initial_state(i["n"], seed=i["seed"])) for i in inst]
        b = [c.new_state() for c in ctxs]
        return ctxs, a, b

    def timed_sweep(mode, steps, warmup, batch_mode=0):
        chnss.set_batch_mode(batch_mode)
        ctxs, a, b = make(mode)
        t_rec = time.perf_counter()
        for _ in range(warmup):                 # the first two steps record the ping-pong graphs
            chnss.step_batched(ctxs, a, b, max_threads=threads)
            a, b = b, a
        torch.cuda.synchronize()
        t_rec = time.perf_counter() - t_rec
        launches0 = ctxs[0].profile_read()["launches"]
        stats0 = chnss.batch_stats()
        sampler = ClockSampler(_device_uuid(torch, local))
        barrier()
        sampler.start()
        t0 = time.perf_counter()
        recs, iters = None, []
        for _ in range(steps):
            _, recs, _ = chnss.step_batched(ctxs, a, b, max_threads=threads)
            iters.append(recs)
            a, b = b, a
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        barrier()
        clocks = sampler.stop()
        launches = ctxs[0].profile_read()["launches"] - launches0
        stats1 = chnss.batch_stats()
        batch_calls = {k: stats1[k] - stats0[k] for k in stats1}
        if world > 1:
            t = torch.tensor([sec], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            sec = float(t.item())
        conv = all(r[k]["converged"] for rs in iters for r in rs for k in r)
        mean = {k: round(sum(r[k]["iters"] for rs in iters for r in rs) / (len(iters) * len(recs)), 2) for k in recs[0]}
        final = [chnss.state_to_numpy(x) for x in a]
        del ctxs, a, b
        chnss.set_batch_mode(0)
        return sec, clocks, launches, conv, mean, t_rec, final, batch_calls

    sec_g, clocks, launches, conv_g, iters_g, rec_g, fin_g, batch_g = timed_sweep(1, args.sweep_steps, args.warmup)
    value = len(all_inst) * args.sweep_steps / sec_g
    one_graph = None
    if args.sweep_batch_graph_steps > 0:
        sec_b, _, _, conv_b, _, rec_b, _, batch_b = timed_sweep(1, args.sweep_batch_graph_steps, args.warmup, 1)
        one_graph = {"value": round(len(all_inst) * args.sweep_batch_graph_steps / sec_b, 3),
                     "unit": "instance steps/s", "steps": args.sweep_batch_graph_steps, "converged": conv_b,
                     "batch_calls": batch_b, "graph_recording_s": round(rec_b, 2),
                     "how": "chnss_set_batch_mode(1): the whole batch recorded as one CUDA graph (every "
                            "instance's step a parallel branch), one launch per batch step"}
    host = None
    if args.sweep_host_steps > 0:
        sec_h, _, _, conv_h, iters_h, _, fin_h, _ = timed_sweep(0, args.sweep_host_steps, args.warmup)
        host = {"value": round(len(all_inst) * args.sweep_host_steps / sec_h, 3), "unit": "instance steps/s",
                "steps": args.sweep_host_steps, "converged": conv_h, "iters_mean": iters_h,
                "how": "the same batch with host-driven Krylov loops: chnss_step_batched on "
                       f"{threads} worker threads, serial solve groups inside each instance"}
        if args.sweep_host_steps == args.sweep_steps:
            host["equal_final_states"] = all(all(np.array_equal(x[k], y[k]) for k in x) for x, y in zip(fin_g, fin_h))

    # the FP64 step of every instance, one instance at a time (host-driven)
    ctx64, a64, b64 = make(0, lambda i: dict(i["params"], precision=0, ortho=0))
    for c, x, y in zip(ctx64, a64, b64):       # one warm-up step each
        c.step(x, y)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c, x, y in zip(ctx64, b64, a64):
        c.step(x, y)
        c.stream.synchronize()
    seq64 = len(inst) / (time.perf_counter() - t0)
    del ctx64, a64, b64
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    out = {
        "metric": SWEEP_METRIC, "value": round(value, 3), "unit": "instance steps/s", "n_gpus": world,
        "steps": args.sweep_steps, "warmup": args.warmup, "ms_per_step": round(sec_g / args.sweep_steps * 1e3, 3),
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
        "dtype": "f64 outer / f32 preconditioner", "data": "synthetic (seeded SplitMix64 draws)",
        "config": {"workload": f"sweep{len(all_inst)}", "instances": len(all_inst),
                   "instances_rank0": len(inst), "parallelism": f"instances sharded over {world} GPU(s)",
                   "meshes": {str(n): sum(1 for i in all_inst if i["n"] == n)
                              for n in sorted({i["n"] for i in all_inst})},
                   "total_p1_nodes": sum((i["n"] + 1) ** 2 for i in all_inst),
                   "evap_rate": [round(min(i["params"]["evap_rate"] for i in all_inst), 4),
                                 round(max(i["params"]["evap_rate"] for i in all_inst), 4)],
                   "step": ("every instance's step a branch of one recorded CUDA graph, one launch per batch "
                            "step (Krylov loops as conditional nodes)" if batch_g["one_graph"] == args.sweep_steps
                            else "one recorded CUDA graph per instance step (Krylov loops as conditional nodes)"),
                   "batch_calls": batch_g,
                   "gram_schmidt": "double-FP32",
                   "l2": "inputs larger than L2 (tens of GB resident)",
                   "timing": "wall clock around chnss_step_batched (it returns after every stream is synchronised)"},
        "graph_recording_s": round(rec_g, 2),
        "tuning": {str(n): {"block_p1": t["block_p1"], "block_p2": t["block_p2"],
                            "ms_p1": [round(x, 4) for x in t["ms_p1"]], "ms_p2": [round(x, 4) for x in t["ms_p2"]]}
                   for n, t in tuning.items()},
        "one_graph_batch": one_graph,
        "host_driven_batch": host,
        "fp64_one_at_a_time": {"value": round(seq64, 3), "unit": "instance steps/s",
                               "how": "rank 0: the FP64 step (FP64 Gram-Schmidt) of each instance, one after the "
                                      "other, host-driven"},
        "speedup_vs_fp64_one_at_a_time": round(value / world / seq64, 3),
        "converged": conv_g,
        "iters_mean": iters_g,
        "gpu_launches": launches,
        "clocks": clocks,
    }
    print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
def oracle_calibration():
    """A measured full-size oracle step (profiles/oracle_step1024.json, one
    step of the 1024 x 1024 bench parameter set on one host core of the GPU
    machine), against which the node-ratio scaling of the samples is
    checked."""
    try:
        with open(os.path.join(ROOT, "profiles", "oracle_step1024.json")) as f:
            d = json.load(f)
        return {"n": d["n"], "seconds_per_step": d["seconds"][0], "steps_per_s": 1.0 / d["seconds"][0],
                "iters": d.get("iters"), "source": "profiles/oracle_step1024.json"}
    except Exception:
        return None


def run_reference(args):
    """The oracle (plain numpy/scipy FP64, one thread) on the bench workload.
    A full 1024 x 1024 oracle step takes minutes, so each timed step is a
    bounded sample: one oracle step of the same parameter set on a
    REF_SAMPLE_N x REF_SAMPLE_N mesh; the metric (steps/s at 1024 x 1024) is
    that rate scaled by the node ratio, checked against a measured
    full-size step (oracle_calibration)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2501_11767_gb300 import inputs
    n = inputs.workload(args.workload)["n"]
    smp = run_cpu_sample_subprocess(REF_SAMPLE_N, args.workload, steps=args.warmup + args.steps)
    secs = smp["seconds"][args.warmup:]
    sec = sum(secs) / len(secs)
    scale = nodes(REF_SAMPLE_N) / nodes(n)
    value = scale / sec
    calib = oracle_calibration()
    sample = (f"each timed step is one oracle step (numpy/scipy FP64, 1 thread) of the same parameter set on a "
              f"{REF_SAMPLE_N}x{REF_SAMPLE_N} mesh ({nodes(REF_SAMPLE_N)} nodes, {sec:.2f} s); value = that rate "
              f"x the node ratio {nodes(REF_SAMPLE_N)}/{nodes(n)}")
    out = {
        "impl": "reference", "metric": workload_metric(args.workload, n, inputs.workload(args.workload)["params"]),
        "value": value, "unit": "steps/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(sec * 1e3, 1),
        "ms_per_step_is": f"wall time of one sampled {REF_SAMPLE_N}x{REF_SAMPLE_N} oracle step",
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "n": n, "sampled_n": REF_SAMPLE_N,
                   "scaled_to_n_by": "node ratio"},
        "cpu_baseline": {"value": value, "unit": "steps/s", "cores": 1, "kind": "oracle", "sample": sample,
                         "cpu": cpu_model(), "iters": smp["iters"]},
        "calibration": calib,
        "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    if calib:
        out["calibration"]["scaled_sample_over_measured"] = round(value / calib["steps_per_s"], 3)
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--bf16-steps", type=int, default=5)
    ap.add_argument("--roofline-steps", type=int, default=3)
    ap.add_argument("--ortho", type=int, default=-1, choices=[-1, 0, 1],
                    help="Gram-Schmidt arithmetic of the headline leg: 0 FP64, 1 double-FP32 (-1: the workload's)")
    ap.add_argument("--step-mode", type=int, default=0, choices=[0, 1],
                    help="0: host-driven Krylov loops; 1: every step one recorded CUDA graph")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--sweep", action="store_true", help="batched 64-instance parameter sweep instead")
    ap.add_argument("--adjoint", action="store_true", help="40-step gradient on 256x256 instead")
    ap.add_argument("--three-d", action="store_true", help="the 3D step on a Kuhn mesh instead")
    ap.add_argument("--amg", action="store_true", help="smoothed-aggregation AMG on the 1024^2 CH block instead")
    ap.add_argument("--three-d-n", type=int, default=32)
    ap.add_argument("--nvtx-step", action="store_true",
                    help="with --three-d: one serial mixed step inside an NVTX range (profiling), no timing")
    ap.add_argument("--three-d-mobility", type=int, default=0, choices=[0, 1],
                    help="3D workload with the concentration-dependent mobility")
    ap.add_argument("--three-d-open", type=int, default=0, choices=[0, 1], help="3D workload with an open top")
    ap.add_argument("--three-d-inner", type=float, default=0.0,
                    help="3D workload with multigrid blocks iterated to this tolerance")
    ap.add_argument("--sweep-count", type=int, default=64)
    ap.add_argument("--sweep-threads", type=int, default=0)
    ap.add_argument("--sweep-concurrent-steps", action="store_true")
    ap.add_argument("--sweep-steps", type=int, default=50, help="steps of every instance in the timed sweep")
    ap.add_argument("--sweep-batch-graph-steps", type=int, default=10,
                    help="steps of the same sweep as one graph launch per batch step (0: skip)")
    ap.add_argument("--sweep-host-steps", type=int, default=5,
                    help="steps of the host-driven comparison batch (0: skip)")
    ap.add_argument("--cpu-sample", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--cpu-steps", type=int, default=1, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours" and not args.cpu_sample:
        ap.error("--warmup must be >= 3")
    if args.cpu_sample:
        print(json.dumps(cpu_sample(args.cpu_sample, args.workload, args.cpu_steps)))
        return
    if args.impl == "reference":
        run_reference(args)
        return
    if args.sweep:
        run_sweep(args)
        return
    if args.adjoint:
        run_adjoint(args)
        return
    if args.three_d:
        run_three_d(args)
        return
    if args.amg:
        run_amg(args)
        return
    run_gpu(args)


if __name__ == "__main__":
    main()
