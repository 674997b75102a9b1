#!/usr/bin/env python3
"""Benchmark of the R-SLB shock-tube step on GB300.

Workload: the ultrarelativistic Sod shock tube at scale -- 65536 cells on
[-1, 1], 3 x 200 velocities (Gauss-Laguerre x Gauss-Legendre), N_Omega = 5,
CFL 0.5, outflow boundaries -- for each relaxation time tau in
{1e-4, 1e-2, 1, 10}.  One bench step = one TVD-RK3 time step (three fused
stage kernels) of each of the four tubes, FP32 populations with FP64 Landau
matching.  Metric: cell-velocity updates per second.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank advances its own replica of the workload
(the single-tube step has no exchange to shard), rank 0 prints one JSON line.
"""
import argparse
import hashlib
import re
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1612_01287_gb300 import workloads  # noqa: E402

METRIC = "cell-velocity updates/s"
UNIT = "cv-updates/s"
TAUS = workloads.SOD_LARGE_TAUS
FALLBACK_HBM_GBS = 6800.0
BYTES_PER_CV_STEP_F32 = 32  # stage 1 r+w (8 B), stages 2-3 read f_n, f^(i), write (12 B each)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tubes", type=int, default=len(TAUS),
                    help="number of the four tau tubes per step (profiling runs use 1)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 side measurement")
    ap.add_argument("--no-side", action="store_true",
                    help="skip the batched Bjorken and batched shock-tube side measurements")
    ap.add_argument("--bj-steps", type=int, default=20)
    ap.add_argument("--bj-runs", type=int, default=16384,
                    help="runs of the batched Bjorken side measurement")
    ap.add_argument("--bj-modes", default="simt,tf32x3",
                    help="contraction modes of the batched Bjorken side measurement")
    ap.add_argument("--only", choices=["bjorken", "sod_batch", "closure"],
                    help="run just this side measurement and print its JSON (profiling)")
    ap.add_argument("--batch-steps", type=int, default=10)
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x, dist, device):
    """The slowest rank's time (every rank gets it); x itself without a process group."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, units_per_rank, seconds):
    """Units all ranks processed (each rank its own replica) per second of the
    slowest rank."""
    return world * units_per_rank / seconds


def workload_dt(w):
    from paper_1612_01287_gb300 import quadrature
    xi, _, _, _ = quadrature(w["Q_xi"], w["Q_L"])
    return w["cfl"] * w["dz"] / float(np.abs(xi).max())


def oracle_workload_dt(w):
    """The same time step from the oracle's own Gauss-Legendre nodes (the CPU
    legs depend on oracle/ alone)."""
    import oracle
    xi, _ = oracle.gauss_legendre(w["Q_xi"])
    return w["cfl"] * w["dz"] / float(np.abs(xi).max())


def config_dict(w, dt, ntubes=len(TAUS)):
    taus = ",".join("%g" % t for t in TAUS[:ntubes])
    return {"workload": "sod_shock_tube_Nx%d_NL%d_Nxi%d_tau{%s}" % (
        w["Z"], w["Q_L"], w["Q_xi"], taus),
        "cells": w["Z"], "velocities": w["Q_L"] * w["Q_xi"], "N_Omega": w["N_Omega"],
        "dt": dt, "cfl": w["cfl"], "tubes_per_step": ntubes, "bc": w["bc"],
        "precision": "fp32 populations, fp64 Landau matching",
        "l2": "inputs larger than L2 (157 MB per population buffer)"}


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples every 50 ms; stop() keeps those taken inside the window
    marked by region_begin()/region_end() (all of them if none falls inside)."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(prefix="rslb_clocks_", suffix=".csv")
            self.fh = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=timestamp,clocks.sm,clocks.max.sm,power.draw,"
                 "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def region_begin(self):
        self.t0 = time.time()

    def region_end(self):
        self.t1 = time.time()

    @staticmethod
    def parse(lines, t0=None, t1=None):
        """Summary of nvidia-smi CSV lines (timestamp first); samples outside
        [t0, t1] are dropped when some fall inside."""
        import datetime
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rec = (float(parts[1]), float(parts[2]), parts[5:9])
            except ValueError:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                ts = None
            rows.append((ts, rec))
        inside = [r for ts, r in rows
                  if t0 is not None and t1 is not None and ts is not None and t0 <= ts <= t1]
        use = inside if inside else [r for _, r in rows]
        if not use:
            return None
        reasons = set()
        for _, _, flags in use:
            for n, v in zip(names, flags):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(r[0] for r in use), "sm_max_mhz": max(r[1] for r in use),
                "samples": len(use), "in_timed_region": bool(inside), "reasons": sorted(reasons)}

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        out = self.parse(open(self.path), self.t0, self.t1)
        try:
            os.remove(self.path)
        except OSError:
            pass
        return out


# --------------------------------------------------------------------------- helpers
def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            for k in ("hbm_gbs", "hbm_GBs", "hbm"):
                if k in d:
                    return float(d[k]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


KERNEL_SOURCES = {
    # the sources a stage kernel is compiled from
    "sod32_stage_kernel": ("paper_1612_01287_gb300/csrc/sod32.cu",
                           "paper_1612_01287_gb300/csrc/sod32_core.cuh",
                           "paper_1612_01287_gb300/csrc/sod.cuh",
                           "paper_1612_01287_gb300/csrc/rslb_device.cuh", "include/rslb.h"),
}
KERNEL_SOURCES["sod_stage_kernel<double,8>"] = KERNEL_SOURCES["sod_stage_kernel<double,16>"] = (
    "paper_1612_01287_gb300/csrc/sod.cu", "paper_1612_01287_gb300/csrc/sod.cuh",
    "paper_1612_01287_gb300/csrc/rslb_device.cuh")
# of these headers the kernel uses only the lines that match
KERNEL_SOURCE_LINES = {"include/rslb.h": re.compile(r"^#define RSLB_PACKED_TILE_CELLS\b")}


def source_sha(kernel="sod32_stage_kernel"):
    h = hashlib.sha256()
    files = KERNEL_SOURCES.get(kernel)
    if files is None:
        csrc = os.path.join(ROOT, "paper_1612_01287_gb300", "csrc")
        files = [os.path.join("paper_1612_01287_gb300", "csrc", f) for f in sorted(os.listdir(csrc))]
    for f in files:
        text = open(os.path.join(ROOT, f), encoding="utf-8").read()
        pat = KERNEL_SOURCE_LINES.get(f)
        if pat is not None:
            text = "".join(l for l in text.splitlines(True) if pat.match(l))
        h.update(" ".join(_strip_comments(text).split()).encode())
    return h.hexdigest()[:16]


def _strip_comments(text):
    """C/C++ source without its comments (the recorded traffic follows the
    code, not the prose; the caller also collapses white space); string
    literals are kept as they are."""
    out, i, n = [], 0, len(text)
    while i < n:
        ch = text[i]
        if ch == '"':
            j = i + 1
            while j < n and text[j] != '"':
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(ch)
            i += 1
    return "".join(out)


def recorded_traffic(kernel):
    """DRAM bytes per launch from the last ncu capture, if the kernel source is unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path)).get(kernel)
        if d and d.get("source_sha") == source_sha(kernel):
            return d.get("dram_bytes_per_launch")
    except Exception:
        pass
    return None


def recorded_fp64_ops(kernel):
    """FP64-pipe lane operations per cell-velocity and stage of an FP64 stage
    kernel, from the last ncu count, if the kernel source is unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(path)).get(kernel)
        if d and d.get("source_sha") == source_sha(kernel):
            return d.get("fp64_lane_ops_per_cv_stage")
    except Exception:
        pass
    return None


HBARC_GEV_FM = 0.1973269804
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # SMs x FP32 lanes x FMA x max SM clock


def measured_tf32_peak():
    """Dense TF32 tensor peak: the measured BF16 GEMM burst rate times the nominal
    TF32/BF16 ratio 1/2 (1.1 vs 2.25 PFLOP/s); None without the measurement."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(path))["bf16_tflops"]) / 2.0
    except Exception:
        return None


def _timed(stream, fn, n):
    import torch
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    fn(n)
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b)


def bench_bjorken(stream, steps=None):
    """Batched Bjorken flow: 16384 runs, Q_xi integer-uniform in [8, 512], Q_L = 3,
    eta/s log-uniform [0.01, 10], T0 uniform [0.3, 0.6] GeV, tau0 = 0.5 fm/c
    (nondimensional tau from 1), dtau = 1e-3.  One step = one RK3 step of every run."""
    from paper_1612_01287_gb300 import Bjorken
    steps = steps or ARGS.bj_steps
    qxi, eta_s, T0 = workloads.bjorken_batch(nruns=ARGS.bj_runs)
    taus = 5 * HBARC_GEV_FM * eta_s / (0.5 * T0)
    cv = 3 * int(qxi.sum())
    q = qxi.astype(np.float64)
    # the method's contraction K^P f as a dense product: 2 Q^2 flops per radial
    # column, 3 columns per run, 3 RK stages per step
    flops = 3 * 2 * 3 * float((q ** 2).sum())
    # what the tensor cores execute: the even (ceil(Q/2)^2) and odd (floor(Q/2)^2)
    # half-size products, three TF32 products each (hi.hi, hi.lo, lo.hi)
    qh, h = np.ceil(q / 2), np.floor(q / 2)
    pipe_flops = 3 * 3 * 2 * 3 * float((qh ** 2 + h ** 2).sum())
    out = {"runs": len(qxi), "cv_per_step": cv, "kp_flops_per_step": flops,
           "tensor_pipe_flops_per_step": pipe_flops}
    for mode in ARGS.bj_modes.split(","):
        with Bjorken(qxi, "parton", taus, Q_L=3, precision="f32", kp_mode=mode, dtau=1e-3,
                     stream=stream) as b:
            b.step(1)
            ms = _timed(stream, b.step, steps) / steps
            o = b.read()
            if not np.all(np.isfinite(o["E"])):
                raise RuntimeError("non-finite Bjorken state")
        out[mode] = {"value": cv / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
                     "steps": steps, "kp_tflops": flops / (ms * 1e-3) / 1e12,
                     "fp32_peak_tflops": FP32_PEAK_TFLOPS}
        if mode == "tf32x3":
            # the contraction as a tensor-core roofline: three TF32 products per
            # FP32 product (hi.hi, hi.lo, lo.hi) against the dense TF32 peak
            peak = measured_tf32_peak()
            pipe = pipe_flops / (ms * 1e-3) / 1e12
            useful = flops / (ms * 1e-3) / 1e12
            out[mode]["tensor_roofline"] = {
                "bound": "tensor", "achieved": pipe, "unit": "TFLOP/s",
                "peak": peak, "frac": pipe / peak if peak else None,
                "peak_source": "measured bf16 x 1/2" if peak else None,
                "useful_tflops": useful, "useful_frac": useful / peak if peak else None,
                "note": "achieved counts the TF32 products the tensor pipe executes (three per "
                        "FP32 product, half-size even/odd matrices); useful counts the dense "
                        "FP32 product K^P f once"}
    return out


def bench_sod_batch(stream, steps=None):
    """Uneven batch of 4096 shock tubes (Z log-uniform [256, 8192], Q_xi in
    {8, 20, 50, 100, 200}, Q_L = 3, tau log-uniform [1e-4, 10], pressure ratio
    [2, 20]); FP32.  Timed (1) over the first batch steps, when every run is
    active, and (2) from the start until the runs have done a tenth of all
    their cell-velocity updates to t_end (runs with few steps finish on the way).
    Beside it, 16 runs of the sweep (seeded sample) to t_end as a batch and one
    at a time through rslb_init/rslb_step (the plain form)."""
    from paper_1612_01287_gb300 import Sod, SodBatch
    steps = steps or ARGS.batch_steps
    runs = workloads.sod_sweep()
    t0 = time.perf_counter()
    peak, _ = measured_peak()
    with SodBatch(runs, precision="f32", autotune=True, stream=stream) as b:
        init_s = time.perf_counter() - t0
        V = np.array([3 * r["Q_xi"] for r in runs], dtype=np.float64)
        Zr = np.array([r["Z"] for r in runs], dtype=np.float64)
        nst = np.array([b.run_info(i)[0] for i in range(len(runs))], dtype=np.float64)
        cv = float((Zr * V).sum())
        b.step(1)
        ms = _timed(stream, b.step, steps) / steps
        tuning = b.tuning()
        total = b.total_cv_updates
        # (2) to a tenth of the work: the batch steps k with
        # sum_r min(k, nsteps_r) Z_r V_r >= total / 10
        done1 = steps + 1
        k = done1
        while float((np.minimum(k, nst) * Zr * V).sum()) < 0.1 * total:
            k += 100
        span = k - done1
        ms_span = _timed(stream, b.step, span)
        cv_span = float((np.minimum(k, nst) * Zr * V).sum() - (np.minimum(done1, nst) * Zr * V).sum())
        m = b.moments(0)
        if not np.all(np.isfinite(m["E"])):
            raise RuntimeError("non-finite batched state")
    rate = cv_span / (ms_span * 1e-3)
    ach = rate * BYTES_PER_CV_STEP_F32 / 1e9
    out = {"runs": len(runs), "value": cv / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
           "steps": steps, "cv_per_step": cv, "init_s": init_s,
           "tuning": [{"V": V_, "tile_cells": B, "ctas_per_sm": K} for V_, B, K in tuning],
           "cv_updates_to_t_end": total,
           "to_tenth_of_work": {"batch_steps": [done1, k], "max_steps": int(nst.max()),
                                "cv_updates": cv_span, "seconds": ms_span * 1e-3,
                                "value": rate, "unit": UNIT,
                                "roofline": {"bound": "hbm", "achieved": ach, "peak": peak,
                                             "unit": "GB/s", "frac": ach / peak,
                                             "bytes_per_cv_update": BYTES_PER_CV_STEP_F32}}}
    # batch against one run at a time, on a sample of the sweep
    rng = np.random.default_rng(workloads.SEED + 1)
    sample = [runs[i] for i in rng.choice(len(runs), size=16, replace=False)]
    with SodBatch(sample, precision="f32", autotune=True, stream=stream) as b:
        b.step(1)
        import torch
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.run_to_end()
        b.moments(0)
        t_batch = time.perf_counter() - t0
        sample_cv = b.total_cv_updates
        info = [b.run_info(i) for i in range(len(sample))]
    t_plain = 0.0
    for r, (n, dtr) in zip(sample, info):
        with Sod(Z=r["Z"], Q_xi=r["Q_xi"], Q_L=3, precision="f32", bc="outflow", tau=r["tau"],
                 dt=dtr, left=(r["nL"], r["TL"], 0.0), right=(r["nR"], r["TR"], 0.0),
                 stream=stream) as s:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.step(int(n))
            s.sync()
            t_plain += time.perf_counter() - t0
    out["batch_vs_plain_sample"] = {
        "runs": len(sample), "cv_updates": sample_cv, "batch_s": t_batch, "plain_s": t_plain,
        "speedup": t_plain / t_batch,
        "note": "the same 16 runs to t_end: one batch (first step excluded) against one "
                "handle per run stepped through rslb_step, one after another"}
    return out


def bench_closure(stream):
    """Learned closure (Q_xi = 8 + MLP) against the plain method.  Shock tube at
    65536 cells to t = 0.05 (3277 steps).  Training: one snapshot from each of 16
    Q_xi = 200 runs with tau log-uniform in [1e-3, 10] (seeded) at a seeded time,
    65536 cell samples each (1.05e6), targets scaled per tau (closure_train).
    Judged at tau in {0.01, 0.1, 0.5, 1}: L2 errors of e and beta against
    Q_xi = 200 on the same grid and their wall times, and the equal-error row: the
    smallest plain Q_xi whose errors are at most 1e-3 and its wall time."""
    import torch
    from paper_1612_01287_gb300 import Sod
    from paper_1612_01287_gb300 import closure_train as CT
    QL, QHI, QLO = 3, 200, 8
    Z, t_end, thr = 65536, 0.05, 1e-3
    dt = 0.5 * (2.0 / Z) / 0.9999306
    nsteps = int(round(t_end / dt))
    rng = np.random.default_rng(workloads.SEED)
    taus = 10.0 ** rng.uniform(-3.0, 1.0, size=16)
    steps = [[int(s)] for s in rng.integers(0, nsteps, size=16)]
    t0 = time.perf_counter()
    X, T, snaps = CT.generate(Z, taus, steps, dt, stream=stream)
    torch.cuda.synchronize()
    out = {"samples": int(X.shape[0]), "datagen_s": time.perf_counter() - t0, "cells": Z,
           "t_end": t_end, "steps": nsteps, "train_taus": [float(t) for t in taus],
           "network": "73-64-64-24 SiLU, BF16 weights, FP32 accumulate; targets scaled per tau"}
    t0 = time.perf_counter()
    cl_model, losses = CT.train(X, T, snaps, epochs=40, batch=8192, lr=2e-3, stream=stream)
    out["train_s"] = time.perf_counter() - t0
    out["loss_first_last"] = [float(losses[0]), float(losses[-1])]
    out["explained_by_log10_tau"] = [[round(float(x), 3), round(float(y), 3)]
                                     for x, y in zip(*cl_model.explained)]
    del X, T

    def l2(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))

    def run(q, tau, closure=False):
        with Sod(Z=Z, Q_xi=q, Q_L=QL, N_Omega=min(q - 1, 5), precision="f32", bc="outflow",
                 tau=tau, dt=dt, stream=stream) as s:
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            if closure:
                cl_model.step(s, tau, nsteps)
            else:
                s.step(nsteps)
            m = s.moments()
            return m, time.perf_counter() - t1

    acc = {}
    with cl_model:
        for tau in (0.01, 0.1, 0.5, 1.0):
            try:
                mh, t_hi = run(QHI, tau)
                ml, t_lo = run(QLO, tau)
                mc, t_cl = run(QLO, tau, closure=True)
                err = lambda m: {"e": l2(m["E"], mh["E"]), "beta": l2(m["beta"], mh["beta"])}
                row = {"closure_active": cl_model.active(tau),
                       "plain_q8": err(ml), "closure_q8": err(mc),
                       "wall_s": {"q200_plain": t_hi, "q8_plain": t_lo, "q8_closure": t_cl}}
                ok = lambda e: e["e"] <= thr and e["beta"] <= thr
                eq = {"threshold": thr, "closure_reaches": ok(row["closure_q8"]),
                      "plain_q8_reaches": ok(row["plain_q8"])}
                for q in (8, 12, 16, 24, 32, 48, 64, 100, 150):
                    if q == QLO:
                        e, tq = row["plain_q8"], t_lo
                    else:
                        mq, tq = run(q, tau)
                        e = err(mq)
                    if ok(e):
                        eq.update({"plain_q_needed": q, "plain_wall_s": tq, "plain_err": e})
                        break
                if eq["closure_reaches"]:
                    eq["closure_wall_s"] = t_cl
                row["equal_error"] = eq
                acc[str(tau)] = row
            except Exception as exc:
                acc[str(tau)] = {"error": repr(exc)[:200]}
        out["l2_vs_q200"] = acc
        # per-step cost at this size
        with Sod(Z=Z, Q_xi=QHI, Q_L=QL, N_Omega=5, precision="f32", bc="outflow", tau=1.0,
                 dt=dt, stream=stream) as hi, \
                Sod(Z=Z, Q_xi=QLO, Q_L=QL, N_Omega=5, precision="f32", bc="outflow", tau=1.0,
                    dt=dt, stream=stream) as cl:
            hi.step(2)
            cl_model.step(cl, 1.0, 2)
            ms_hi = _timed(stream, hi.step, 8) / 8
            ms_cl = _timed(stream, lambda k: cl_model.step(cl, 1.0, k), 8) / 8
    out["ms_per_step_65536"] = {"q200_plain": ms_hi, "q8_closure": ms_cl,
                                "speedup": ms_hi / ms_cl}
    return out


def _oracle_window(job):
    """One process of a CPU leg: the FP64 oracle advances `cells` cells of one tube
    (tau = 1e-2, all velocities; the window starts at cell `lo`, outflow ends) by
    `warmup` untimed and `steps` timed RK3 steps; returns the timed seconds."""
    w, lo, cells, dt, steps, warmup = job
    import oracle
    dz = w["dz"]
    zc = -1.0 + (np.arange(lo, lo + cells) + 0.5) * dz
    (nL, TL, bL), (nR, TR, bR) = w["left"], w["right"]
    p = oracle.sod_params(cells, w["Q_xi"], w["Q_L"], w["N_Omega"], z_min=-1.0 + lo * dz,
                          z_max=-1.0 + (lo + cells) * dz, bc="outflow", tau_mode="const",
                          tau=1e-2, dt=dt)
    f = oracle.sod_init_fields(p, np.where(zc < 0, nL, nR), np.where(zc < 0, TL, TR),
                               np.where(zc < 0, bL, bR))
    if warmup:
        f = oracle.sod_steps(p, f, warmup)
    t0 = time.perf_counter()
    oracle.sod_steps(p, f, steps)
    return time.perf_counter() - t0


def oracle_rate(w, dt, procs, cells, steps, warmup=0):
    """Cell-velocity updates/s of the single-threaded oracle run in `procs`
    processes at once (spawned: this may run after CUDA work), each on its own
    window of `cells` cells around the membrane; the slowest process sets the
    time.  Returns (rate, slowest seconds, cell-velocity updates)."""
    import multiprocessing as mp
    Z = w["Z"]
    first = Z // 2 - procs * cells // 2
    jobs = [(w, first + i * cells, cells, dt, steps, warmup) for i in range(procs)]
    if procs == 1:
        times = [_oracle_window(jobs[0])]
    else:
        with mp.get_context("spawn").Pool(procs) as pool:
            times = pool.map(_oracle_window, jobs)
    cvu = procs * cells * w["Q_xi"] * w["Q_L"] * steps
    el = max(times)
    return cvu / el, el, cvu


def cpu_baseline(w, steps=20):
    """The FP64 oracle on the host cores, on bounded samples of the workload: one
    process on 1024 cells, then one process per core, each on its own 512-cell
    window around the membrane (the same single-threaded code; windows are
    independent problems with outflow ends)."""
    dt = oracle_workload_dt(w)
    ncores = os.cpu_count() or 1
    V = w["Q_xi"] * w["Q_L"]
    one, el1, _ = oracle_rate(w, dt, 1, 1024, steps)
    allc, elc, cvc = oracle_rate(w, dt, ncores, 512, steps)
    return {"value": allc, "unit": UNIT, "cores": ncores, "kind": "oracle",
            "sample": "%d processes (one per core) x 512 cells x %d velocities x %d RK3 steps "
                      "of one tube (tau=1e-2), single-threaded FP64 C oracle in each, %.1f s "
                      "wall" % (ncores, V, steps, elc),
            "single_thread": {"value": one, "unit": UNIT, "cores": 1,
                              "sample": "1024 cells x %d velocities x %d RK3 steps, %.1f s"
                                        % (V, steps, el1)}}


# --------------------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    """The oracle, as it stands, on all host cores: one process per core, each
    advancing its own 512-cell window of the tau = 1e-2 tube by one RK3 step per
    bench step (W untimed, K timed).  Depends on oracle/ alone."""
    if rank != 0:
        return 0
    w = workloads.sod_large()
    dt = oracle_workload_dt(w)
    ncores = os.cpu_count() or 1
    cells = 512
    val, el, _ = oracle_rate(w, dt, ncores, cells, args.steps, warmup=args.warmup)
    sample = ("%d processes (one per core) x %d cells x %d velocities, one RK3 step per "
              "bench step, single-threaded FP64 C oracle in each" % (ncores, cells,
                                                                   w["Q_xi"] * w["Q_L"]))
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(w, dt),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": ncores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- our arm
def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1612_01287_gb300 import Sod, build
    torch.cuda.set_device(local_rank)
    build.build()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    w = workloads.sod_large()
    dt = workload_dt(w)
    # a dedicated stream: the library captures its RK steps into a CUDA graph
    # on non-default streams
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    # each tube on its own stream: the tubes are independent, so their stage
    # kernels may overlap (one tube's launches fill the last waves of another's)
    ntubes = max(1, min(args.tubes, len(TAUS)))
    tstreams = [torch.cuda.Stream() for _ in range(ntubes)]
    tubes = [Sod(Z=w["Z"], Q_xi=w["Q_xi"], Q_L=w["Q_L"], N_Omega=w["N_Omega"], bc=w["bc"],
                 tau=tau, dt=dt, left=w["left"], right=w["right"], precision="f32",
                 stream=ts) for tau, ts in zip(TAUS[:ntubes], tstreams)]
    V, Z = w["Q_xi"] * w["Q_L"], w["Z"]
    cv_per_step = V * Z * len(tubes)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        for t in tubes:
            t.step(1)
    barrier()
    # per-launch timing of the stage kernels: the tubes one after another, one
    # event pair per tube-step on the tube's stream, each tube-step waiting for
    # the previous one, so no two launches overlap
    pairs, prev = [], None
    for _ in range(args.steps):
        for t, ts in zip(tubes, tstreams):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            if prev is not None:
                ts.wait_event(prev)
            a.record(ts)
            t.step(1)
            b.record(ts)
            pairs.append((a, b))
            prev = b
    barrier()
    per_tube_step_ms = [a.elapsed_time(b) for a, b in pairs]
    # the timed region: every tube's steps, the tubes concurrently
    clk = ClockSampler(local_rank)
    clk.start()
    time.sleep(0.3)
    barrier()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    clk.region_begin()
    start.record(stream)
    for ts in tstreams:
        ts.wait_event(start)
    for _ in range(args.steps):
        for t in tubes:
            t.step(1)
    for ts in tstreams:
        e = torch.cuda.Event()
        e.record(ts)
        stream.wait_event(e)
    end.record(stream)
    barrier()
    clk.region_end()
    clocks = clk.stop()
    ms = start.elapsed_time(end)
    ms = max_over_ranks(ms, dist, "cuda")
    for t in tubes:
        t.sync()

    # ---- end to end through the C ABI with host buffers ----
    # the same tubes, each on a handle with its own stream, so that the copy
    # of one tube's populations overlaps the RK step of another.  Per step and
    # tube: pinned host populations -> device (rslb_set_state), one RK3 step
    # (rslb_step); then the 14 fields of every tube -> pinned host
    # (rslb_moments, which waits for its tube's stream).
    host_f, host_m = [], []
    for t in tubes:
        hf = torch.empty(V * Z, dtype=torch.float32).pin_memory()
        hf.copy_(torch.from_numpy(t.get_state().reshape(-1)))
        host_f.append(hf)
        host_m.append(torch.empty(14 * Z, dtype=torch.float64).pin_memory())
    e_streams = [torch.cuda.Stream() for _ in tubes]
    e_tubes = [Sod(Z=w["Z"], Q_xi=w["Q_xi"], Q_L=w["Q_L"], N_Omega=w["N_Omega"], bc=w["bc"],
                   tau=tau, dt=dt, left=w["left"], right=w["right"], precision="f32",
                   stream=es) for tau, es in zip(TAUS[:len(tubes)], e_streams)]
    nbytes = V * Z * 4

    def e2e_run(nsteps):
        # every step of every tube: copy in, step, read the fields back; a
        # tube's next step is queued as soon as its fields of this step are
        # back, so the tubes do not wait for one another between steps
        for t, hf in zip(e_tubes, host_f):
            t.set_state_ptr(hf.data_ptr(), 0)
            t.step(1)
        for k in range(nsteps):
            for t, hf, hm in zip(e_tubes, host_f, host_m):
                t.moments_into(hm.data_ptr())
                if k + 1 < nsteps:
                    t.set_state_ptr(hf.data_ptr(), 0)
                    t.step(1)

    e2e_run(2)  # warm-up
    e2e_steps = max(1, min(args.e2e_steps, args.steps))
    barrier()
    t0 = time.perf_counter()
    e2e_run(e2e_steps)
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, dist, "cuda")
    e2e_val = whole_job_rate(world, cv_per_step * e2e_steps, e2e_s)
    for t in e_tubes:
        t.close()

    # ---- FP64 path, one tube, a few steps (ALU-bound on this part) ----
    fp64 = None
    if rank == 0 and not args.no_fp64:
        with Sod(Z=w["Z"], Q_xi=w["Q_xi"], Q_L=w["Q_L"], N_Omega=w["N_Omega"], bc=w["bc"],
                 tau=1e-2, dt=dt, left=w["left"], right=w["right"], precision="f64",
                 stream=stream) as t64:
            t64.step(1)
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            t64.step(2)
            b.record(stream)
            torch.cuda.synchronize()
            fms = a.elapsed_time(b) / 2
            from paper_1612_01287_gb300._lib import measure_fp64_fma
            dfma = measure_fp64_fma(20, stream)
            fp64 = {"value": V * Z / (fms * 1e-3), "unit": UNIT, "ms_per_tube_step": fms,
                    "note": "one tube, FP64 everywhere; bound by the FP64 pipe, not HBM",
                    "measured_dfma_per_s": dfma}
            k64 = "sod_stage_kernel<double,%d>" % t64.launch_info()[0]
            ops = recorded_fp64_ops(k64)
            if ops:
                # FP64 lane operations the kernel executes (ncu, per cell-velocity and
                # stage) against the measured DFMA lane rate: the FP64-pipe roofline
                ach = ops * V * Z * 3 / (fms * 1e-3)
                fp64["roofline"] = {"bound": "fp64", "achieved": ach / 1e9, "peak": dfma / 1e9,
                                    "unit": "G FP64 lane-ops/s", "frac": ach / dfma,
                                    "ops_per_cv_stage": ops, "kernel": k64,
                                    "note": "FP64 lane operations (DFMA + DADD + DMUL, ncu) "
                                            "per cell-velocity and stage against the "
                                            "measured DFMA lane rate"}

    B_tile = tubes[0].launch_info()[0]
    from paper_1612_01287_gb300._lib import PACKED_TILE_CELLS
    kname = ("sod32_stage_kernel" if B_tile == PACKED_TILE_CELLS
             else "sod_stage_kernel<float,%d>" % B_tile)
    for t in tubes:
        t.close()
    extras = {}
    if rank == 0 and not args.no_side:
        for name, fn in (("bjorken", bench_bjorken), ("sod_batch", bench_sod_batch),
                         ("closure", bench_closure)):
            try:
                extras[name] = fn(stream)
            except Exception as exc:  # a side measurement never sinks the headline line
                extras[name] = {"error": repr(exc)[:300]}
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    value = whole_job_rate(world, cv_per_step * args.steps, ms * 1e-3)
    per_launch_ms = statistics.mean(per_tube_step_ms) / 3.0
    peak, peak_kind = measured_peak()
    achieved = BYTES_PER_CV_STEP_F32 / 3.0 * V * Z / (per_launch_ms * 1e-3) / 1e9
    achieved_conc = BYTES_PER_CV_STEP_F32 * cv_per_step / (ms / args.steps * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config_dict(w, dt, len(tubes)),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": peak_kind,
                     "kernel": kname,
                     "algorithmic_bytes_per_launch": BYTES_PER_CV_STEP_F32 / 3.0 * V * Z,
                     "avg_launch_ms": per_launch_ms,
                     "traffic": recorded_traffic(kname),
                     # the timed region itself (tubes concurrent): all launches'
                     # algorithmic bytes over its length
                     "achieved_concurrent": achieved_conc,
                     "frac_concurrent": achieved_conc / peak},
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": nbytes * len(tubes),
                "d2h_bytes_per_step": 14 * Z * 8 * len(tubes), "steps": e2e_steps,
                "note": "per step, for each tube on its own stream: pinned host populations "
                        "-> device (rslb_set_state), one RK3 step (rslb_step), 14 fields -> "
                        "pinned host (rslb_moments); a tube's next step is queued when its "
                        "fields are back"},
        "schedule": "each tube on its own CUDA stream in the timed region; the roofline's "
                    "launch times come from a pass with the tubes one after another",
        "gpu_launches": 3 * len(tubes) * args.steps,
        "clocks": clocks,
        "fp64": fp64,
    }
    line.update(extras)
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(w)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


ARGS = None


def main():
    global ARGS
    args = parse()
    ARGS = args
    rank, world, local_rank = dist_env()
    if args.only:
        import torch
        from paper_1612_01287_gb300 import build
        build.build()
        torch.cuda.set_device(local_rank)
        stream = torch.cuda.Stream()
        torch.cuda.set_stream(stream)
        fn = {"bjorken": bench_bjorken, "sod_batch": bench_sod_batch,
              "closure": bench_closure}[args.only]
        print(json.dumps({args.only: fn(stream)}), flush=True)
        return 0
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
