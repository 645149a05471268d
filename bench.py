#!/usr/bin/env python
"""Benchmark: 256^3 Poisson-lognormal MAP solve on one GB300.

A step is one whole MAP solve (every part of the hot path): from s = mu,
Newton-Krylov iterations (FP64 gradient of Sec. 3.1.2 through the 3D FFT
prior, FP32 Jacobi-preconditioned CG on the Hessian, step length of
Eq. New5, Armijo line search) until ||g|| / ||g0|| < 1e-6, on the production
workload: 256^3 cells, 500 Mpc/h box, sigma_G = 1.8, nbar = 1, w = 1, a
512-bin P(k) table; synthetic lognormal-Poisson counts (seed 1 + rank).

Printed as one JSON line.  `value` is MAP solves per second over all ranks
(inputs resident in HBM); `e2e` the same with the counts copied in from
pinned host memory and the MAP copied out inside each step (the copies of
neighbouring steps overlap the solve on a second stream).  Extra keys:
time-to-MAP of the mixed and the FP64 forms, Hessian-vector products per
second (FP32, FP64), per-kernel device time and the roofline of the
dominant kernel, and the FP64 CPU oracle timed on a bounded sample.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl plc|reference]
    python bench.py --cpu-full [--out FILE]

With --impl reference the FP64 CPU oracle is timed instead (rank 0 only).
--cpu-full times whole oracle solves on the host cores (minutes: the 256^3
solve alone takes several) and measures the mixed-precision GPU MAP against
the oracle's MAP converged to 1e-12; its record, committed under profiles/,
is quoted in the default line with the sources it was taken on.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("256³ time-to-MAP (‖g‖/‖g0‖<1e-6) & Hv/s; mixed vs FP64 GPU, "
          "HBM frac")
UNIT = "MAP/s"
WORKLOAD = "production256"
TOL = 1e-6
# Work of one FP64 Newton-Krylov MAP solve of this workload, used to scale
# the oracle's timed sample (one Hv, one gradient + objective) to MAP/s.  The
# oracle takes the FP64 GPU solve's steps (12 Newton steps, 31 CG iterations,
# 13 gradient evaluations with the line-search trials); it applies one more
# Hv per Newton step for xi^T H xi of Eq. (New5) and evaluates every trial
# through the FFT: 31 + 12 = 43 Hv and 13 gradient + objective evaluations.
REF_HV_PER_MAP = 43
REF_GRAD_PER_MAP = 13


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (out or "").splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------
# algorithmic bytes per launch of each kernel kind inside the mixed MAP solve
# ----------------------------------------------------------------------------
def algorithmic_bytes(n: int) -> dict:
    """Bytes each kernel kind must move per launch in the mixed MAP solve."""
    n3, h = n ** 3, n // 2 + 1
    spec32, spec64 = 8 * h * n * n, 16 * h * n * n
    return {
        # FP32 Hessian-vector product of the CG, direction update fused in
        "xf_f32": 4 * 4 * n3 + spec32,          # read r, D, p; write p; write spectrum
        "yf_f32": 2 * spec32, "z_f32": 2 * spec32, "yi_f32": 2 * spec32,
        "xi_f32": spec32 + 3 * 4 * n3,          # read spectrum, D, p; write Hp
        # FFT gradients (w = 1): read s, write the spectrum; read the
        # spectrum, s, N, write y, D, r (FP32 phase: all FP32, no g, which
        # the trial forms again from y, D and N) or y, g, D, r (FP64 context,
        # y and g in FP64)
        "grad_xf_f32": 4 * n3 + spec32,
        "grad_yf_f32": 2 * spec32, "grad_z_f32": 2 * spec32, "grad_yi_f32": 2 * spec32,
        "grad_xi_f32": spec32 + (4 + 4 + 3 * 4) * n3,
        "grad_xf_f64": 8 * n3 + spec64,
        "grad_yf_f64": 2 * spec64, "grad_z_f64": 2 * spec64, "grad_yi_f64": 2 * spec64,
        "grad_xi_f64": spec64 + (8 + 4 + 4 * 8) * n3,
        # read x, p, r, Hp, D; write x, r (the first iteration of a solve
        # writes x = alpha p without reading x: 4 bytes less, see main)
        "cg_update_f32": 7 * 4 * n3,
        # line-search trial: read xi, r, D, s, y, N; write s, y, D, r (the
        # FP32 phase keeps no g); FP64 phase: also read and write g
        "newton_update_f32": (6 * 4 + 4 * 4) * n3,
        "newton_update_f64": (3 * 4 + 3 * 8 + 4 + 3 * 8 + 2 * 4) * n3,
    }


def bias_bytes(n: int) -> dict:
    """Algorithmic bytes per launch of the linear-bias model's FP32 passes,
    averaged over the three pipelines of its CG product (B(E p) -> Q .,
    B(.) -> E ., S^-1 p + d1 p + .): the mix of nearly all its launches."""
    n3, h = n ** 3, n // 2 + 1
    spec = 8 * h * n * n
    return {"bias_xf_f32": (28 * n3 + 3 * spec) / 3, "bias_yf_f32": 2 * spec,
            "bias_z_f32": 2 * spec, "bias_yi_f32": 2 * spec,
            "bias_xi_f32": (32 * n3 + 3 * spec) / 3, "cg_update_f32": 7 * 4 * n3}


def dominant_kernel(ctx, run, nbytes: dict) -> dict:
    """Run `run()` once with per-launch CUDA events on (`run` should enqueue
    one CG iteration per chunk, so that no launch is an early exit that would
    pull the mean down); the kernel kind with
    the most device time, its mean duration and, where its algorithmic bytes
    per launch are known, the achieved bandwidth against the measured peak."""
    ctx.profile_enable(True)
    run()
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    tot = sum(v[2] for v in prof.values())
    k, (nl, nt, ms) = max(prof.items(), key=lambda kv: kv[1][2])
    avg_us = 1e3 * ms / nt if nt else None
    out = {"kernel": k, "share": ms / tot if tot else None, "avg_us": avg_us, "launches": nl}
    if k in nbytes and avg_us:
        gbs = nbytes[k] / (avg_us * 1e-6) / 1e9
        out.update({"achieved_gbs": gbs, "frac": gbs / peaks()[0], "peak": "measured hbm_gbs"})
    return out


def fft_flops(n: int) -> float:
    """5 N log2 N per complex line transform of length n."""
    return 5.0 * n * math.log2(n)


def algorithmic_flops_f64(n: int) -> dict:
    h = n // 2 + 1
    lines_x, lines_yz = n * n / 2, h * n
    f = {"xf_f64": lines_x * fft_flops(n), "yf_f64": lines_yz * fft_flops(n),
         "z_f64": 2 * lines_yz * fft_flops(n), "yi_f64": lines_yz * fft_flops(n),
         "xi_f64": lines_x * fft_flops(n)}
    f.update({"grad_" + k: v for k, v in list(f.items())})
    return f


FP64_PEAK_TFLOPS = 1.25   # GB300 nominal FP64 rate (no FP64 figure is measured)


def load_traffic(n: int):
    """Per-launch DRAM bytes from the committed ncu summary, if still current."""
    path = os.path.join(ROOT, "profiles", f"dram_traffic_{WORKLOAD}.txt")
    if not os.path.exists(path):
        return {}, None
    from paper_0911_1407_gb300 import build
    src_hash = build.source_hash()
    out, file_hash = {}, None
    for line in open(path):
        line = line.strip()
        if line.startswith("# csrc "):
            file_hash = line.split()[2]
        elif line and not line.startswith("#"):
            k, v = line.split()[:2]
            out[k] = float(v)
    return (out, file_hash) if file_hash == src_hash else ({}, file_hash)


# ----------------------------------------------------------------------------
# the oracle on the host cores
# ----------------------------------------------------------------------------
CPU_RECORD = os.path.join(ROOT, "profiles", "cpu_baseline_oracle.json")


def oracle_hash() -> str:
    """Hash of the oracle's sources (the CPU baseline is the oracle as it stands)."""
    import glob
    import hashlib
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(ROOT, "oracle", "*.py"))):
        h.update(os.path.basename(f).encode())
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def time_oracle_map(spec, warmup: int, reps: int, tol: float = TOL):
    """Whole oracle MAP solves of one workload, s^0 = mu to ||g|| / ||g0|| < tol:
    `warmup` untimed, then `reps` timed; returns the mock, the problem, the
    last result and the timed seconds."""
    from oracle import plc as orc
    from paper_0911_1407_gb300 import mocks
    m = mocks.make_mock(spec)
    p = orc.make_problem(m.N, m.w, m.nbar, m.mu, m.n, m.box, m.k_tab, m.P_tab)
    r, times = None, []
    for k in range(warmup + reps):
        t0 = time.perf_counter()
        r = orc.newton_krylov_map(p, tol=tol)
        if k >= warmup:
            times.append(time.perf_counter() - t0)
    return m, p, r, times


def batch_spec_of_size(n: int):
    from paper_0911_1407_gb300 import mocks
    return next(sp for sp in mocks.batch_specs() if sp.n == n)


def timing_entry(name, m, r, times, warmup):
    return {"workload": name, "n": m.n, "seconds": statistics.median(times),
            "maps_per_s": 1.0 / statistics.median(times), "runs": len(times), "warmup": warmup,
            "newton_iters": r.newton_iters, "cg_iters": r.cg_iters, "grad_rel": r.grad_rel}


def cpu_full(args):
    """Whole oracle solves on the host cores and the mixed GPU MAP against the
    oracle's MAP at 1e-12 (selection128, production256); one JSON record."""
    import torch
    from paper_0911_1407_gb300 import build
    build.build()
    import paper_0911_1407_gb300 as plc
    from paper_0911_1407_gb300 import mocks
    from oracle import plc as orc
    torch.cuda.set_device(0)
    rec = {"csrc": build.source_hash(), "oracle": oracle_hash(), "cores": os.cpu_count(),
           "cpu_model": cpu_model(), "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()),
           "tol": TOL, "timing": "time.perf_counter around oracle.plc.newton_krylov_map, "
                                 "s^0 = mu, median of the timed runs", "time_to_map": [],
           "mixed_vs_oracle": {}}
    plan = [("C1 plain32", mocks.WORKLOADS["plain32"], 1, 3),
            ("C5 64^3 (batch mock)", batch_spec_of_size(64), 1, 3),
            ("C5 96^3 (batch mock)", batch_spec_of_size(96), 1, 3),
            ("C5 128^3 (batch mock)", batch_spec_of_size(128), 0, 3),
            ("C2 selection128", mocks.WORKLOADS["selection128"], 0, 3),
            ("C3 production256", mocks.WORKLOADS["production256"], 0, 1)]
    finals = {}
    for name, spec, warm, reps in plan:
        m, p, r, times = time_oracle_map(spec, warm, reps)
        rec["time_to_map"].append(timing_entry(name, m, r, times, warm))
        print(json.dumps(rec["time_to_map"][-1]), flush=True)
        if spec.name in ("selection128", "production256"):
            finals[spec.name] = (m, p, r)
    def err(a, ref, N):
        d = a - ref
        i = np.unravel_index(int(np.argmax(np.abs(d))), d.shape)
        return {"max_abs": float(np.abs(d[i])),
                "rel_l2": float(np.linalg.norm(d) / np.linalg.norm(ref)),
                "at_max": {"N": int(N[i]), "s_ref": float(ref[i])}}

    for key, (m, p, r) in finals.items():
        # the oracle continued from its 1e-6 iterate to 1e-12 (same g0: the
        # minimiser is unique, so the path does not matter)
        t0 = time.perf_counter()
        ref = orc.newton_krylov_map(p, s0=r.s, g0_norm=r.g0_norm, tol=1e-12)
        t_more = time.perf_counter() - t0
        Nd = torch.from_numpy(m.N).cuda()
        w = None if m.w is None else torch.from_numpy(m.w).cuda()
        out = {"oracle_grad_rel": ref.grad_rel, "oracle_converged": bool(ref.converged),
               "oracle_newton_iters_past_1e-6": ref.newton_iters,
               "oracle_seconds_past_1e-6": t_more,
               # how far a 1e-6 stop is from the MAP, in the oracle itself
               "oracle_tol1e-6": err(r.s, ref.s, m.N)}
        for prec in ("mixed", "fp64"):
            c = plc.Context(m.n, m.box, prec)
            c.set_prior(m.k_tab, m.P_tab, m.mu)
            tols = (TOL, 1e-8, 1e-10) if prec == "mixed" else (TOL,)
            for tol in tols:
                res = c.newton_krylov_map(Nd, w, m.nbar, tol=tol)
                e = err(res.s.cpu().numpy(), ref.s, m.N)
                e["grad_rel"] = res.stats["grad_rel"]
                out[f"{prec}_tol{tol:g}"] = e
            c.close()
        # the headline pair: the mixed MAP at the metric's tolerance
        out["max_abs"] = out[f"mixed_tol{TOL:g}"]["max_abs"]
        out["rel_l2"] = out[f"mixed_tol{TOL:g}"]["rel_l2"]
        rec["mixed_vs_oracle"][key] = out
        print(json.dumps({key: out}), flush=True)
    rec["bias64"] = bias64_vs_oracle(plc, err)
    print(json.dumps({"bias64": rec["bias64"]}), flush=True)
    if args.out:
        os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
        with open(args.out, "w") as f:
            json.dump(rec, f, indent=1)
    print(json.dumps(rec), flush=True)
    return 0


def bias64_vs_oracle(plc, err):
    """The linear-bias MAP on a 64^3 cut of the production workload (500 *
    64 / 256 Mpc/h, sigma_G = 1.8, nbar = 1, b(k) = 1.5 (k / 0.1)^0.1): the
    oracle's own MAP at 1e-6 and converged, and the GPU MAPs against it."""
    import torch
    from oracle import bias as obias, plc as orc
    from paper_0911_1407_gb300 import mocks
    sp = mocks.replace(mocks.WORKLOADS["production256"], n=64, box=125.0)
    m = mocks.make_mock(sp)
    kb, b = mocks.bias_table(m.n, m.box, 1.5, 0.1)
    p = orc.make_problem(m.N, m.w, m.nbar, m.mu, m.n, m.box, m.k_tab, m.P_tab)
    q = obias.BiasProblem(p, obias.bias_multipliers(m.n, m.box, kb, b, 1.5))
    t0 = time.perf_counter()
    r6 = obias.bias_map(q, tol=TOL)
    t6 = time.perf_counter() - t0
    # continue to a gradient 1e-12 of the first g0 (the oracle takes no g0)
    g6 = float(np.linalg.norm(obias.bias_gradient(r6.s, q)))
    ref = obias.bias_map(q, s0=r6.s, tol=max(1e-12 * r6.g0_norm / g6, 1e-8))
    g_ref = float(np.linalg.norm(obias.bias_gradient(ref.s, q))) / r6.g0_norm
    out = {"oracle_seconds_to_1e-6": t6, "oracle_newton_iters_to_1e-6": r6.newton_iters,
           "oracle_grad_rel_converged": g_ref, "oracle_tol1e-6": err(r6.s, ref.s, m.N)}
    Nd = torch.from_numpy(m.N).cuda()
    for prec in ("mixed", "fp64"):
        c = plc.Context(m.n, m.box, prec)
        c.set_prior(m.k_tab, m.P_tab, m.mu)
        c.set_bias(kb, b, 1.5)
        for tol in (TOL, 1e-8):
            s = torch.zeros((m.n,) * 3, dtype=torch.float64, device="cuda")
            res = c.bias_map(Nd, None, m.nbar, s=s, tol=tol)
            e = err(s.cpu().numpy(), ref.s, m.N)
            e.update({"grad_rel": res.stats["grad_rel"], "newton_iters": res.stats["newton_iters"]})
            out[f"{prec}_tol{tol:g}"] = e
        c.close()
    return out


def cpu_record():
    """The committed --cpu-full record, with whether it matches the sources."""
    if not os.path.exists(CPU_RECORD):
        return None
    from paper_0911_1407_gb300 import build
    rec = json.load(open(CPU_RECORD))
    rec["matches_current_csrc"] = rec.get("csrc") == build.source_hash()
    rec["matches_current_oracle"] = rec.get("oracle") == oracle_hash()
    rec["source"] = "profiles/cpu_baseline_oracle.json (python bench.py --cpu-full)"
    return rec


def time_oracle_sample(m, repeats: int = 1):
    """One oracle Hessian-vector product and one gradient at full size."""
    from oracle import plc as orc
    p = orc.make_problem(m.N, m.w, m.nbar, m.mu, m.n, m.box, m.k_tab, m.P_tab)
    s = np.full(m.N.shape, m.mu) + 0.1 * np.random.default_rng(0).standard_normal(m.N.shape)
    v = np.random.default_rng(1).standard_normal(m.N.shape)
    t_hv, t_g = [], []
    for _ in range(repeats):
        t0 = time.perf_counter()
        orc.hessvec(s, v, p)
        t1 = time.perf_counter()
        orc.gradient(s, p)
        orc.neg_log_posterior(s, p)
        t2 = time.perf_counter()
        t_hv.append(t1 - t0)
        t_g.append(t2 - t1)
    return min(t_hv), min(t_g)


def reference_arm(args):
    from paper_0911_1407_gb300 import mocks
    m = mocks.make_mock(mocks.WORKLOADS[WORKLOAD])
    hv_per_map = REF_HV_PER_MAP
    grad_per_map = REF_GRAD_PER_MAP
    for _ in range(args.warmup):
        time_oracle_sample(m)
    times = []
    for _ in range(args.steps):
        t_hv, t_g = time_oracle_sample(m)
        times.append(t_hv * hv_per_map + t_g * grad_per_map)
    t_map = statistics.median(times)
    cores = os.cpu_count()
    sample = (f"one FP64 oracle Hessian-vector product and one gradient+objective at 256^3 per step, "
              f"scaled to one MAP by {hv_per_map} Hv and {grad_per_map} gradients per solve")
    line = {"impl": "reference", "metric": METRIC, "value": 1.0 / t_map, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_map, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.gpus),
            "precision": "FP64 throughout (the oracle)",
            "cpu_baseline": {"value": 1.0 / t_map, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample, "cpu_model": cpu_model()},
            "e2e": {"value": 1.0 / t_map, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    rec = cpu_record()
    if rec is not None:
        # whole oracle solves measured by --cpu-full, beside the modelled figure
        line["cpu_baseline"]["measured_full"] = {
            k: rec.get(k) for k in ("time_to_map", "cores", "cpu_model", "when", "oracle",
                                    "matches_current_oracle", "source")}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# the GPU arm
# ----------------------------------------------------------------------------
# ----------------------------------------------------------------------------
# replicas over ranks (one process per GPU; no data-path collective)
# ----------------------------------------------------------------------------
def workload_config(world: int) -> dict:
    """The `config` of the JSON line, the same for both arms."""
    from paper_0911_1407_gb300 import mocks
    spec = mocks.WORKLOADS[WORKLOAD]
    return {"workload": WORKLOAD, "n": spec.n, "box": spec.box, "sigma_G": spec.sigma_G,
            "nbar": spec.nbar, "w": 1, "pk_bins": spec.nbins, "tol": TOL,
            "parallelism": f"replicas{world}",
            "l2": "inputs larger than L2 (>1 GB touched per solve)"}


def rank_spec(mocks, rank: int):
    """The workload of one rank: the same configuration, its own seed and mock."""
    return mocks.replace(mocks.WORKLOADS[WORKLOAD], seed=1 + rank, mock_id=rank)


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest x over all ranks (a timing: the slowest rank sets the pace)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, steps: int, seconds: float) -> float:
    """Solves per second over all ranks: every rank ran `steps` solves."""
    return world * steps / seconds


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["plc", "reference"], default="plc")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the FP64 solve, Hv/s sweeps and the CPU baseline")
    ap.add_argument("--micro", choices=["hv32", "hv64", "grad32", "grad64", "map32", "map64"],
                    help="profiling aid: run --reps single operator calls at size --n and exit")
    ap.add_argument("--host-driven", action="store_true",
                    help="run every solve with the host driver instead of one graph launch "
                         "(same kernels; for profilers that cannot see into conditional graphs)")
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--cpu-full", action="store_true",
                    help="time whole oracle solves on the host cores and the mixed GPU MAP "
                         "against the oracle at 1e-12; writes one JSON record (minutes)")
    ap.add_argument("--out", help="file for the --cpu-full record")
    args = ap.parse_args(argv)
    if args.micro:
        return micro(args)
    if args.cpu_full:
        return cpu_full(args)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank == 0:
            reference_arm(args)
        return 0
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_0911_1407_gb300 import build
    build.build()
    import paper_0911_1407_gb300 as plc
    from paper_0911_1407_gb300 import mocks

    spec = rank_spec(mocks, rank)
    m = mocks.make_mock(spec)
    n = m.n
    stream = torch.cuda.current_stream()
    ctx = plc.Context(n, m.box, "mixed")
    ctx.set_prior(m.k_tab, m.P_tab, m.mu)
    N_dev = torch.from_numpy(m.N).cuda()
    s = torch.empty((n, n, n), dtype=torch.float64, device="cuda")

    driven = 0 if args.host_driven else 1

    # each solve starts at mu (start=2: the start is the prior mean without
    # an array holding it, so s is output only and needs no fill)
    def step():
        return ctx.newton_krylov_map(N_dev, None, m.nbar, s=s, tol=TOL, start=2,
                                     device_driven=driven)

    # clocks are sampled from the warm-up on (nvidia-smi takes a moment to
    # start), through the end of the timed region: all under load
    clocks = ClockSampler(local)
    clocks.start()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---------------- timed region: K whole MAP solves -----------------------
    ctx.profile_enable(False)            # launch counts only, no per-launch events
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats = [step().stats for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    t_dev = e0.elapsed_time(e1) / 1e3
    # each solve is one graph launch; the library counts the kernels it ran
    # (the host driver's launches are counted by the profiling counters)
    launches = (int(sum(v[0] for v in ctx.profile_read().values())) if args.host_driven
                else int(sum(st["kernels"] for st in stats)))
    t_dev = max_over_ranks(t_dev, world, "cuda")
    value = whole_job_rate(world, args.steps, t_dev)

    # ---------------- second timed region with per-launch CUDA events --------
    # (the events add a little host and device time, so `value` above is
    # taken without them; the kernel durations and the roofline come from here)
    # The per-launch events need the host-driven form of the same solve (a
    # graph cannot hold event records in its loops); it takes the same steps
    # and launches the same kernels.  CG chunks of one iteration, so that no
    # launch is an early exit.
    ctx.profile_enable(True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        ctx.newton_krylov_map(N_dev, None, m.nbar, s=s, tol=TOL, start=2, cg_chunk=1,
                              device_driven=0)
    e1.record(stream)
    torch.cuda.synchronize()
    t_prof = e0.elapsed_time(e1) / 1e3
    prof = ctx.profile_read()
    ctx.profile_enable(False)

    # ---------------- end to end: host buffers in and out --------------------
    # Every step copies its counts in from pinned host memory and its MAP out
    # to pinned host memory.  Two buffer sets alternate and the copies run on
    # a second stream, so that step k+1's counts come in and step k-1's MAP
    # goes out while step k solves (the solve call itself is synchronous).
    N_host = torch.from_numpy(m.N).pin_memory()
    s_host = [torch.empty((n, n, n), dtype=torch.float64).pin_memory() for _ in range(2)]
    N_buf = [N_dev, torch.empty_like(N_dev)]
    s_buf = [s, torch.empty_like(s)]
    copy = torch.cuda.Stream()

    def e2e_run(k_steps):
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_solved = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]
        copy.wait_stream(stream)
        with torch.cuda.stream(copy):
            N_buf[0].copy_(N_host, non_blocking=True)
            ev_in[0].record(copy)
        for k in range(k_steps):
            b = k % 2
            if k + 1 < k_steps:
                # buffer 1-b was read by solve k-1, which has returned
                with torch.cuda.stream(copy):
                    N_buf[1 - b].copy_(N_host, non_blocking=True)
                    ev_in[1 - b].record(copy)
            stream.wait_event(ev_in[b])
            if k >= 2:
                stream.wait_event(ev_out[b])      # step k-2's MAP has left s_buf[b]
            ctx.newton_krylov_map(N_buf[b], None, m.nbar, s=s_buf[b], tol=TOL, start=2,
                                  device_driven=driven)
            ev_solved[b].record(stream)
            with torch.cuda.stream(copy):
                copy.wait_event(ev_solved[b])
                s_host[b].copy_(s_buf[b], non_blocking=True)
                ev_out[b].record(copy)
        stream.wait_stream(copy)

    e2e_run(2)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0.record(stream)
    e2e_run(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    t_e2e = e0.elapsed_time(e1) / 1e3
    t_e2e = max_over_ranks(t_e2e, world, "cuda")

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    # ---------------- per-kernel roofline (dominant kernel) ------------------
    hbm_peak, peak_kind = peaks()
    abytes = algorithmic_bytes(n)
    aflops = algorithmic_flops_f64(n)
    total_ms = sum(v[2] for v in prof.values())
    kernels = {k: {"launches": v[0], "avg_us": 1e3 * v[2] / v[1] if v[1] else None,
                   "share": v[2] / total_ms if total_ms else None}
               for k, v in prof.items() if v[0]}
    # every CG solve starts with x = alpha p, which does not read x
    first_iters = args.steps * stats[-1]["newton_iters"]
    if prof.get("cg_update_f32", (0,))[0]:
        nl = prof["cg_update_f32"][0]
        abytes["cg_update_f32"] -= 4 * n ** 3 * min(first_iters, nl) / nl
    dom = max(prof, key=lambda k: prof[k][2])
    avg_s = prof[dom][2] / prof[dom][1] / 1e3
    traffic, _ = load_traffic(n)
    if dom.endswith("f64") and dom in aflops:
        ach = aflops[dom] / avg_s / 1e12
        roofline = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS,
                    "traffic": traffic.get(dom), "peak_kind": "nominal FP64"}
    else:
        ach = abytes[dom] / avg_s / 1e9
        roofline = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": hbm_peak,
                    "unit": "GB/s", "frac": ach / hbm_peak, "traffic": traffic.get(dom),
                    "peak_kind": peak_kind}
    hbm_kernels = {}
    for k in prof:
        if prof[k][1] and k in abytes and not k.endswith("f64"):
            gbs = abytes[k] / (prof[k][2] / prof[k][1] / 1e3) / 1e9
            hbm_kernels[k] = round(gbs / hbm_peak, 3)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": workload_config(world),
        "precision": "mixed (FP32 FFT/CG, FP64-accurate gradient, FP64 reductions and state)",
        "clocks": clk,
        "e2e": {"value": whole_job_rate(world, args.steps, t_e2e), "unit": UNIT,
                "h2d_bytes_per_step": int(N_host.numel() * 4),
                "d2h_bytes_per_step": int(s_host[0].numel() * 8),
                "overlap": "copies on a second stream, two buffer sets"},
        "gpu_launches": launches,
        "profiled_ms_per_step": 1e3 * t_prof / args.steps,
        "roofline": roofline,
        "hbm_frac_fp32_kernels": hbm_kernels,
        "kernels": kernels,
        "solve": {k: stats[-1][k] for k in ("newton_iters", "cg_iters", "grad_evals",
                                             "grad_ffts", "grad_ffts_fp64", "grad_rel")},
    }

    if not args.no_extras:
        extras(plc, m, ctx, s, N_dev, line, args)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def micro(args):
    """A few calls of one operator on a small synthetic field (for ncu)."""
    import torch
    from paper_0911_1407_gb300 import build
    build.build()
    import paper_0911_1407_gb300 as plc
    from paper_0911_1407_gb300 import mocks
    n, box = args.n, 500.0 * args.n / 256
    A = mocks.amplitude_for_sigma(n, box, 1.8)
    k, P = mocks.pk_table(n, box, A)
    prec = "fp64" if args.micro.endswith("64") else "mixed"
    c = plc.Context(n, box, prec)
    c.set_prior(k, P, -1.62)
    g = torch.Generator(device="cuda").manual_seed(0)
    s = (-1.62 + 0.5 * torch.randn((n,) * 3, generator=g, device="cuda", dtype=torch.float64)).to(c.real)
    v = torch.randn((n,) * 3, generator=g, device="cuda", dtype=torch.float64).to(c.real)
    N = torch.poisson(torch.exp(s.double())).to(torch.int32)
    out = torch.empty_like(v)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    s64 = torch.empty((n,) * 3, dtype=torch.float64, device="cuda")
    for _ in range(args.reps):
        if args.micro.startswith("hv"):
            c.hessvec(s, None, 1.0, v, out)
        elif args.micro.startswith("grad"):
            c.logpost_grad(s, N, None, 1.0, grad=out)
        else:
            s64.fill_(-1.62)
            c.newton_krylov_map(N, None, 1.0, s=s64, tol=1e-6, raise_on_fail=False,
                                device_driven=0 if args.host_driven else 1)
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps({"micro": args.micro, "n": n, "reps": args.reps,
                      "ms_per_call": e0.elapsed_time(e1) / args.reps}))
    return 0


def extras(plc, m, ctx, s_mixed, N_dev, line, args):
    """FP64 time-to-MAP, Hv/s in both precisions, accuracy, CPU oracle."""
    import torch
    n = m.n
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}
    # Hessian-vector products per second through plc_hessvec
    for prec, reps in (("mixed", 200), ("fp64", 20)):
        c = ctx if prec == "mixed" else plc.Context(n, m.box, "fp64")
        if prec == "fp64":
            c.set_prior(m.k_tab, m.P_tab, m.mu)
        sv = s_mixed.to(c.real)
        v = torch.randn((n, n, n), dtype=c.real, device="cuda")
        hv = torch.empty_like(v)
        for _ in range(3):
            c.hessvec(sv, None, m.nbar, v, hv)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            c.hessvec(sv, None, m.nbar, v, hv)
        e1.record(stream)
        torch.cuda.synchronize()
        out[prec] = reps / (e0.elapsed_time(e1) / 1e3)
        if prec == "fp64":
            ctx64 = c
    hv_bytes = 12 * 4 * n ** 3
    line["hv_per_s"] = {"f32": out["mixed"], "f64": out["fp64"],
                        "f32_hbm_frac_12bn3_model": out["mixed"] * hv_bytes / 1e9 / peaks()[0]}
    # FP64 time-to-MAP, and accuracy of the mixed MAP against it
    s64 = torch.full((n, n, n), m.mu, dtype=torch.float64, device="cuda")
    r = ctx64.newton_krylov_map(N_dev, None, m.nbar, s=s64, tol=TOL)    # warm-up
    s64.fill_(m.mu)
    torch.cuda.synchronize()
    e0.record(stream)
    r = ctx64.newton_krylov_map(N_dev, None, m.nbar, s=s64, tol=TOL)
    e1.record(stream)
    torch.cuda.synchronize()
    t64 = e0.elapsed_time(e1) / 1e3
    d = (s_mixed - s64)
    line["time_to_map_s"] = {"mixed": line["ms_per_step"] / 1e3, "fp64": t64}
    line["fp64_solve"] = {k: r.stats[k] for k in ("newton_iters", "cg_iters", "grad_evals",
                                                  "grad_ffts", "grad_rel")}
    # the FP64 form is bound by the FP64 pipe: its dominant kernel against
    # the FP64 rate measured here with cuBLAS DGEMM (4096^3 through
    # torch.matmul; MEASURED_PEAKS.json has no FP64 figure) and the nominal one
    a = torch.randn((4096, 4096), dtype=torch.float64, device="cuda")
    b = torch.randn((4096, 4096), dtype=torch.float64, device="cuda")
    for _ in range(3):
        torch.matmul(a, b)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(5):
        torch.matmul(a, b)
    e1.record(stream)
    torch.cuda.synchronize()
    dgemm = 5 * 2 * 4096 ** 3 / (e0.elapsed_time(e1) * 1e-3) / 1e12
    del a, b
    s64b = torch.empty_like(s64)
    dom = dominant_kernel(ctx64, lambda: ctx64.newton_krylov_map(
        N_dev, None, m.nbar, s=s64b.fill_(m.mu), tol=TOL, device_driven=0, cg_chunk=1),
        {"cg_update_f64": 7 * 8 * n ** 3})
    fl = algorithmic_flops_f64(n).get(dom["kernel"])
    if fl and dom.get("avg_us"):
        ach = fl / (dom["avg_us"] * 1e-6) / 1e12
        dom.update({"achieved_tflops": ach, "frac_of_dgemm": ach / dgemm,
                    "frac_of_nominal": ach / FP64_PEAK_TFLOPS})
    line["fp64_solve"]["dominant"] = dom
    line["fp64_peak_measured"] = {"tflops": dgemm, "how": "cuBLAS DGEMM 4096^3 (torch.matmul)",
                                  "nominal_tflops": FP64_PEAK_TFLOPS}
    line["mixed_vs_fp64"] = {"max_abs": float(d.abs().max()),
                             "rel_l2": float(d.norm() / s64.norm())}
    # the FP32 -> FP64 switch point of the mixed solve
    sweep = {}
    sm = torch.empty_like(s64)
    for sw in (1e-4, 1e-5, 3e-6, 1e-6):
        for rep in range(2):
            sm.fill_(m.mu)
            torch.cuda.synchronize()
            e0.record(stream)
            rs = ctx.newton_krylov_map(N_dev, None, m.nbar, s=sm, tol=TOL, mixed_switch=sw)
            e1.record(stream)
            torch.cuda.synchronize()
        dd = sm - s64
        sweep[f"{sw:g}"] = {"ms": e0.elapsed_time(e1), "newton": rs.stats["newton_iters"],
                            "cg": rs.stats["cg_iters"], "grad_rel": rs.stats["grad_rel"],
                            "max_abs_vs_fp64": float(dd.abs().max())}
    line["mixed_switch_sweep"] = sweep
    # host-driven form of the same solve (host reads scalars per CG chunk)
    for rep in range(2):
        sm.fill_(m.mu)
        torch.cuda.synchronize()
        e0.record(stream)
        ctx.newton_krylov_map(N_dev, None, m.nbar, s=sm, tol=TOL, device_driven=0)
        e1.record(stream)
        torch.cuda.synchronize()
    line["host_driven_ms"] = e0.elapsed_time(e1)
    # the LSQ-Wiener filter on the same data (one CG solve of
    # (S^-1 + diag(nbar w)) delta = N - nbar w)
    lsq = {}
    for prec, cc, tol in (("mixed", ctx, 1e-6), ("fp64", ctx64, 1e-6)):
        d = torch.empty((n, n, n), dtype=torch.float64, device="cuda")
        cc.wiener_lsq(N_dev, None, m.nbar, out=d, tol=tol)
        torch.cuda.synchronize()
        e0.record(stream)
        _, _, st = cc.wiener_lsq(N_dev, None, m.nbar, out=d, tol=tol)
        e1.record(stream)
        torch.cuda.synchronize()
        lsq[prec] = {"ms": e0.elapsed_time(e1), "cg_iters": st["cg_iters"],
                     "rel_residual": st["grad_rel"]}
    lsq["dominant_mixed"] = dominant_kernel(
        ctx, lambda: ctx.wiener_lsq(N_dev, None, m.nbar, tol=1e-6, cg_chunk=1),
        algorithmic_bytes(n))
    line["lsq_wiener"] = lsq
    # the Gaussian-prior Poisson MAP (Eq. MAPG) on the same data, from delta = 0
    dg = torch.zeros((n, n, n), dtype=torch.float64, device="cuda")
    ctx.gauss_map(N_dev, None, m.nbar, delta=dg, tol=TOL)
    dg.zero_()
    torch.cuda.synchronize()
    e0.record(stream)
    rg = ctx.gauss_map(N_dev, None, m.nbar, delta=dg, tol=TOL)
    e1.record(stream)
    torch.cuda.synchronize()
    line["gauss_prior_map"] = {"ms": e0.elapsed_time(e1), "precision": "mixed",
                               **{k: rg.stats[k] for k in ("newton_iters", "cg_iters",
                                                           "grad_ffts", "grad_rel")}}
    dg2 = torch.zeros_like(dg)
    line["gauss_prior_map"]["dominant"] = dominant_kernel(
        ctx, lambda: ctx.gauss_map(N_dev, None, m.nbar, delta=dg2.zero_(), tol=TOL, cg_chunk=1),
        algorithmic_bytes(n))
    bias_extra(plc, m, N_dev, line)
    adjoint_extra(plc, line)
    # reconstruction quality against the true field (r and D_Euc, Sec. 4.1.2)
    # and the matter statistics of ln(1 + delta) after 10 Mpc/h smoothing
    d_true = torch.expm1(torch.from_numpy(m.s_true).cuda())
    ests = {"lognormal_map": torch.expm1(s_mixed), "gauss_prior_map": dg,
            "lsq_wiener": ctx.wiener_lsq(N_dev, None, m.nbar, tol=1e-6)[0],
            "inverse_weighting": N_dev.double() / m.nbar - 1.0}
    quality = {}
    for name, d in ests.items():
        corr, de = ctx.compare(d, d_true)
        quality[name] = {"r": corr, "d_euc": de}
    sm = torch.empty_like(d_true)
    for name, d in (("truth", d_true), ("lognormal_map", ests["lognormal_map"])):
        ctx.smooth(d, 10.0, out=sm)
        _, outside, mom = ctx.log_stats(sm, -4.0, 0.2, 40)
        quality.setdefault(name, {})["smoothed10"] = {
            "mean": mom[0], "var": mom[1], "skewness": mom[2], "kurtosis": mom[3],
            "invalid": outside[2]}
    # timings after the calls above (first launches load the kernels): CUDA
    # events around each synchronising call, the mean of 5
    def timed(fn, reps=5):
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps
    t_cmp = timed(lambda: ctx.compare(ests["lognormal_map"], d_true))
    t_smooth = timed(lambda: ctx.smooth(d_true, 10.0, out=sm))
    t_stats = timed(lambda: ctx.log_stats(sm, -4.0, 0.2, 40))
    quality["ms"] = {"compare": t_cmp, "smooth": t_smooth, "log_stats": t_stats}
    # plc_compare reads two FP64 fields (16 B/cell)
    quality["compare_hbm_frac"] = 16 * n ** 3 / (t_cmp * 1e-3) / 1e9 / peaks()[0]
    line["reconstruction_quality"] = quality
    batch_extra(plc, line)
    # the FP64 oracle on the host cores, on a bounded sample
    if int(os.environ.get("WORLD_SIZE", "1")) == 1:
        t_hv, t_g = time_oracle_sample(m)
        # the oracle's own iteration on this workload (as the reference arm)
        hvc, gc = REF_HV_PER_MAP, REF_GRAD_PER_MAP
        t_map = t_hv * hvc + t_g * gc
        # whole oracle solves that fit the bounded budget, measured here:
        # C1 (32^3) and one 64^3 batch mock, median of 3 after 1 warm-up
        measured = []
        for name, spec in (("C1 plain32", mocks_mod().WORKLOADS["plain32"]),
                           ("C5 64^3 (batch mock)", batch_spec_of_size(64))):
            mm, _, rr, times = time_oracle_map(spec, 1, 3)
            measured.append(timing_entry(name, mm, rr, times, 1))
        line["cpu_baseline"] = {
            "value": 1.0 / t_map, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "cpu_model": cpu_model(),
            "sample": (f"modelled: one oracle Hv ({t_hv:.2f} s) and one gradient+objective "
                       f"({t_g:.2f} s) at 256^3, scaled to the oracle's {hvc} Hv and {gc} "
                       f"gradients per MAP; measured: whole oracle solves of C1 and a 64^3 "
                       f"mock in this run (measured_here), and of every config in the "
                       f"committed --cpu-full record (measured_full)"),
            "hv_per_s": 1.0 / t_hv, "measured_here": measured}
        rec = cpu_record()
        if rec is not None:
            line["cpu_baseline"]["measured_full"] = {
                k: rec.get(k) for k in ("time_to_map", "cores", "cpu_model", "when", "oracle",
                                        "matches_current_oracle", "source")}
    rec = cpu_record()
    if rec is not None:
        line["mixed_vs_oracle"] = {**rec.get("mixed_vs_oracle", {}), "csrc": rec.get("csrc"),
                                   "matches_current_csrc": rec["matches_current_csrc"],
                                   "source": rec["source"]}


def mocks_mod():
    from paper_0911_1407_gb300 import mocks
    return mocks


def bias_extra(plc, m, N_dev, line):
    """The linear-bias MAP (Sec. 2.4.1) on the same counts, from delta_M = 0,
    with the scale-dependent table b(k) = 1.5 (k / 0.1 h/Mpc)^0.1: time to
    MAP in both precisions and the kernel shares of one host-timed solve."""
    import torch
    from paper_0911_1407_gb300 import mocks
    n = m.n
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kb, b = mocks.bias_table(n, m.box, 1.5, 0.1)
    out = {"table": "b(k) = 1.5 (k / 0.1 h/Mpc)^0.1, b_dc = 1.5"}
    s = torch.zeros((n, n, n), dtype=torch.float64, device="cuda")
    for prec, reps in (("mixed", 2), ("fp64", 1)):
        c = plc.Context(n, m.box, prec)
        c.set_prior(m.k_tab, m.P_tab, m.mu)
        c.set_bias(kb, b, 1.5)
        for _ in range(reps):
            s.zero_()
            torch.cuda.synchronize()
            e0.record(stream)
            r = c.bias_map(N_dev, None, m.nbar, s=s, tol=TOL)
            e1.record(stream)
            torch.cuda.synchronize()
        out[prec] = {"ms": e0.elapsed_time(e1),
                     **{k: r.stats[k] for k in ("newton_iters", "cg_iters", "grad_evals",
                                                "grad_ffts", "grad_ffts_fp64", "grad_rel",
                                                "kernels")}}
        if prec == "mixed":
            s_bias = s.clone()
            c.profile_enable(True)
            s.zero_()
            # one CG iteration per chunk: no launch is an early exit
            c.bias_map(N_dev, None, m.nbar, s=s, tol=TOL, cg_chunk=1)
            prof = c.profile_read()
            c.profile_enable(False)
            tot = sum(v[2] for v in prof.values())
            top = sorted(((k, v) for k, v in prof.items() if v[0]), key=lambda kv: -kv[1][2])[:8]
            out["kernel_shares"] = {k: {"launches": v[0], "ms": round(v[2], 3),
                                        "share": round(v[2] / tot, 3)} for k, v in top}
            k0, v0 = top[0]
            nb = bias_bytes(n).get(k0)
            if nb and v0[1]:
                avg_us = 1e3 * v0[2] / v0[1]
                gbs = nb / (avg_us * 1e-6) / 1e9
                out["dominant"] = {"kernel": k0, "avg_us": avg_us, "achieved_gbs": gbs,
                                   "frac": gbs / peaks()[0], "bytes": "CG-product mix average"}
        if prec == "mixed":
            ctx_mixed = c
        else:
            c.close()
    d = s_bias - s
    out["mixed_vs_fp64"] = {"max_abs": float(d.abs().max()), "rel_l2": float(d.norm() / s.norm())}
    # At 1e-6 the gradient does not pin s in the voids of this model to 1e-4
    # (the oracle's own 1e-6 stop is ~1e-4 from its converged MAP on a 64^3
    # cut): the two precisions compared again at 1e-8, where it does.
    s8m = torch.zeros_like(s)
    r8m = ctx_mixed.bias_map(N_dev, None, m.nbar, s=s8m, tol=1e-8)
    c64 = plc.Context(n, m.box, "fp64")
    c64.set_prior(m.k_tab, m.P_tab, m.mu)
    c64.set_bias(kb, b, 1.5)
    s8 = torch.zeros_like(s)
    r8 = c64.bias_map(N_dev, None, m.nbar, s=s8, tol=1e-8)
    d8 = s8m - s8
    out["tol1e-8"] = {"mixed_vs_fp64": {"max_abs": float(d8.abs().max()),
                                        "rel_l2": float(d8.norm() / s8.norm())},
                      "mixed_newton_iters": r8m.stats["newton_iters"],
                      "fp64_newton_iters": r8.stats["newton_iters"],
                      "fp64_1e-6_vs_fp64_1e-8_max_abs": float((s - s8).abs().max())}
    ctx_mixed.close()
    c64.close()
    line["bias_map"] = out


def adjoint_extra(plc, line):
    """C4: the MAP and its implicit adjoint at 128^3 (adjoint128): forward
    solve, plc_map_vjp for a cotangent (one CG solve on H lam = u), and the
    same through the autograd function MapField (forward + backward)."""
    import torch
    from paper_0911_1407_gb300 import autograd, mocks
    m = mocks.make_mock(mocks.WORKLOADS["adjoint128"])
    n = m.n
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    N_dev = torch.from_numpy(m.N).cuda()
    u = torch.randn((n, n, n), dtype=torch.float64, device="cuda",
                    generator=torch.Generator(device="cuda").manual_seed(2))
    out = {}
    for prec in ("mixed", "fp64"):
        c = plc.Context(n, m.box, prec)
        c.set_prior(m.k_tab, m.P_tab, m.mu)
        s = torch.full((n, n, n), m.mu, dtype=torch.float64, device="cuda")
        c.newton_krylov_map(N_dev, None, m.nbar, s=s, tol=TOL)
        vtol = 1e-6 if prec == "mixed" else 1e-10
        c.map_vjp(s, None, m.nbar, u, tol=vtol)
        torch.cuda.synchronize()
        e0.record(stream)
        _, _, st = c.map_vjp(s, None, m.nbar, u, tol=vtol)
        e1.record(stream)
        torch.cuda.synchronize()
        out[prec] = {"vjp_ms": e0.elapsed_time(e1), "cg_iters": st["cg_iters"],
                     "rel_residual": st["grad_rel"], "tol": vtol}
        c.close()
    # autograd: forward MAP + backward adjoint through torch.autograd
    c = plc.Context(n, m.box, "mixed")
    Nf = N_dev.double().requires_grad_(True)
    lnA = torch.zeros((), dtype=torch.float64, device="cuda", requires_grad=True)
    for rep in range(2):
        torch.cuda.synchronize()
        e0.record(stream)
        s_map = autograd.map_field(Nf, lnA, c, m.k_tab, m.P_tab, m.mu, None, m.nbar, tol=TOL)
        (s_map * u).sum().backward()
        e1.record(stream)
        torch.cuda.synchronize()
    out["autograd_forward_backward_ms"] = e0.elapsed_time(e1)
    c.close()
    line["adjoint128"] = out


def batch_extra(plc, line):
    """64 independent mocks of uneven sizes (16 x 64^3, 32 x 96^3, 16 x 128^3,
    sigma_G ~ U[0.8, 1.8], nbar log-uniform in [0.2, 2]), mixed precision, to
    ||g|| / ||g0|| < 1e-6: one graph launch for all against one device-driven
    solve after another on one stream."""
    import torch
    from paper_0911_1407_gb300 import mocks
    ms = [mocks.make_mock(sp) for sp in mocks.batch_specs()]
    cs = []
    for m in ms:
        c = plc.Context(m.n, m.box, "mixed")
        c.set_prior(m.k_tab, m.P_tab, m.mu)
        cs.append(c)
    # FFT schedule per grid size: autotuned on the first context of each size
    schedules = {}
    for c in cs:
        if c.n not in schedules:
            f1, f2, us = c.autotune(reps=20)
            schedules[c.n] = {"f1": f1, "f2": f2, "us_per_hv": us}
        c.set_fft_schedule(schedules[c.n]["f1"], schedules[c.n]["f2"])
    Ns = [torch.from_numpy(m.N).cuda() for m in ms]
    ss = [torch.empty((m.n,) * 3, dtype=torch.float64, device="cuda") for m in ms]
    nb = [m.nbar for m in ms]
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def one_by_one():
        for c, m, N, s in zip(cs, ms, Ns, ss):
            s.fill_(m.mu)
            c.newton_krylov_map(N, None, m.nbar, s=s, tol=TOL)

    b = plc.Batch(cs)

    def batched():
        for m, s in zip(ms, ss):
            s.fill_(m.mu)
        return b.map(Ns, None, nb, ss, tol=TOL)

    times = {}
    for name, fn in (("one_by_one", one_by_one), ("batched", batched)):
        fn()                      # captures the graphs
        torch.cuda.synchronize()
        best = None
        for _ in range(3):
            e0.record(stream)
            out = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / 1e3
            best = t if best is None else min(best, t)
        times[name] = best
    _, stats = out
    line["batch"] = {
        "mocks": len(ms), "sizes": "16x64^3, 32x96^3, 16x128^3", "precision": "mixed", "tol": TOL,
        "maps_per_s_batched": len(ms) / times["batched"],
        "maps_per_s_one_by_one": len(ms) / times["one_by_one"],
        "speedup": times["one_by_one"] / times["batched"],
        "newton_iters": sum(st["newton_iters"] for st in stats),
        "cg_iters": sum(st["cg_iters"] for st in stats),
        "kernels": sum(st["kernels"] for st in stats),
        "max_grad_rel": max(st["grad_rel"] for st in stats),
        "fft_schedules": {str(k): v for k, v in schedules.items()}}
    del b, cs


if __name__ == "__main__":
    sys.exit(main())
