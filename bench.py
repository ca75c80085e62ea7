#!/usr/bin/env python
"""Benchmark of the GB300 variational-embedding solver (Algorithm 6 of arXiv:2106.02682).

One step = one sweep of the translation-invariant ADMM / projected dual ascent over the whole
instance (pair pass, rho_0 update, dual updates, block DFT, per-wavevector projection, inverse
DFT).  Default workload: 1-D transverse-field Ising chain, h = 1, 2-spin clusters (16 x 16 pair
marginals), 4096 clusters = 4096 wavevectors (8192 spins), float64.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|df64|mixed]
                    [--workload NAME] [--impl ours|reference] [--no-ttb]

Prints one JSON line (rank 0).  For N > 1 (torchrun) every rank runs its own replica of the
instance (the sweep has no cross-instance exchange); value = sweeps of all ranks / max time.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-certified-bound (residual 1e-6) & ADMM iter/s, warm vs plain, 1 GB300"
UNIT = "iter/s"
FP64_PEAK_TFLOPS = 1.25        # nominal GB300 FP64 (152 SMs x 2 FP64 FMA/clk x 2.07 GHz x 2)
FP32_PEAK_TFLOPS = 80.5        # 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz
L2_FLUSH_BYTES = 512 << 20     # > 129 MB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="tfim1d_L2_N4096")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed", "df64"])
    ap.add_argument("--no-ttb", action="store_true", help="skip the time-to-certified-bound runs")
    ap.add_argument("--ttb-workload", default="tfim1d_L2_N50",
                    help="instance of the time-to-certified-bound runs (default: the paper's TFI "
                         "100x1 table instance, 2x1 clusters, h = 1)")
    ap.add_argument("--ttb-max-iter", type=int, default=40000)
    ap.add_argument("--ttb-max-iter-headline", type=int, default=60000,
                    help="sweep cap of the time-to-certified-bound runs on the benchmark workload")
    ap.add_argument("--ttb-batch", type=int, default=8,
                    help="held-out instances in the batched time-to-bound comparison")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ------------------------------------------------------------------ nvidia-smi clock sampling
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
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
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 8:
                    continue
                try:
                    rows.append((float(parts[0]), float(parts[1]), parts[4:8]))
                except ValueError:
                    continue
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = sorted(r[0] for r in rows)
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for r in rows for i in range(4) if r[2][i].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ algorithmic work per stage
def stage_work(N, D, npass, ncanon):
    """Algorithmic flops / bytes per launch of each stage (float64 words).

    Projection of a real symmetric D x D matrix: tridiagonalisation 4/3 D^3 + back-transform
    2 D^3 + reconstruction D^3 = 13/3 D^3 flops (fixed, whatever eigensolver runs); a complex
    Hermitian one costs 4x that.  The pair pass adds ~60 D^2 elementwise flops per offset.
    A DFT pass reads and writes N * D^2 / 2 complex words.
    """
    P = N - 1
    fs = 13.0 / 3.0 * D ** 3
    return {
        "pair": {"flops": P * (fs + 60 * D * D), "bytes": P * 8 * (6 * D * D + 4 * D)},
        "xproj": {"flops": ncanon * 4 * fs, "bytes": 2 * N * D * D * 8},
        "fft_forward": {"bytes": N * D * D * 8 * 2, "flops": 5.0 * N * D * D / 2 * 6},
        "fft_inverse": {"bytes": N * D * D * 8 * 2, "flops": 5.0 * N * D * D / 2 * 6},
    }


# The translation units the Algorithm-6 kernels of the ncu records are compiled from.
KERNEL_SOURCES = ("ve_bound.cu", "ve_df64.cuh", "ve_device.cuh", "ve_fft.cu", "ve_sweep.cu")


def source_digest(files=KERNEL_SOURCES):
    """Digest of kernel sources with comments and blank lines removed: it changes with the code
    the ncu summaries were taken on, not with its comments."""
    import re
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2106_02682_gb300", "csrc")
    for f in sorted(files):
        with open(os.path.join(csrc, f), encoding="utf-8") as fh:
            text = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
        code = [ln.split("//", 1)[0].rstrip() for ln in text.splitlines()]
        h.update(f.encode())
        h.update("\n".join(ln for ln in code if ln.strip()).encode())
    return h.hexdigest()[:16]


def ncu_record(kernel, workload, precision):
    """The committed ncu record of `kernel` (DRAM traffic per launch, pipe utilisation), if it
    was taken on the current sources; else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as fh:
            data = json.load(fh)
    except (OSError, ValueError):
        return None
    rec = data.get(f"{workload}/{precision}/{kernel}")
    if not rec or rec.get("source_digest") != source_digest():
        return None
    return rec


# ------------------------------------------------------------------ replica aggregation
def job_rate(local_ms, steps, world, device="cpu"):
    """Whole-job sweeps per second for `world` replicas: every rank ran `steps` sweeps, the
    job took as long as the slowest rank (max over ranks of the local device time)."""
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    max_ms = float(t.item())
    return world * steps / (max_ms / 1e3), max_ms


# ------------------------------------------------------------------ CPU oracle timing
def oracle_rate(workload, seconds, max_sweeps=None):
    import numpy as np  # noqa: F401
    from oracle import models as mo
    from oracle import ve_oracle as vo
    from paper_2106_02682_gb300 import synth
    w = synth.WORKLOADS[workload]
    dim = len(w["lattice"])
    terms = mo.tfim_terms(1.0, w["h"], dim) if w["kind"] == "tfim" else mo.xxz_terms(1.0, w["h"], dim)
    pb = vo.Problem(mo.cluster_model(w["lattice"], w["cluster"], *terms))
    vo.set_threads(os.cpu_count() or 1)  # the sweep's independent projections on every host core
    st = vo.initial_state(pb)
    vo.iterate(pb, st)  # warm-up sweep
    n, t0, c0 = 0, time.perf_counter(), time.process_time()
    while True:
        vo.iterate(pb, st)
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds or (max_sweeps and n >= max_sweeps):
            break
    cores = (time.process_time() - c0) / el
    return n / el, n, el, round(cores, 2)


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import models as mo  # noqa: F401
    from oracle import ve_oracle as vo
    from paper_2106_02682_gb300 import synth
    w = synth.WORKLOADS[args.workload]
    dim = len(w["lattice"])
    terms = (mo.tfim_terms(1.0, w["h"], dim) if w["kind"] == "tfim" else mo.xxz_terms(1.0, w["h"], dim))
    pb = vo.Problem(mo.cluster_model(w["lattice"], w["cluster"], *terms))
    vo.set_threads(os.cpu_count() or 1)  # the sweep's independent projections on every host core
    st = vo.initial_state(pb)
    for _ in range(args.warmup):
        vo.iterate(pb, st)
    t0, c0 = time.perf_counter(), time.process_time()
    for _ in range(args.steps):
        vo.iterate(pb, st)
    el = time.perf_counter() - t0
    cores = round((time.process_time() - c0) / el, 2)
    value = args.steps / el
    cfg = workload_config(args, pb.N, pb.D)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": cfg,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} full sweeps of {args.workload} after "
                                   f"{args.warmup} warm-up sweeps (numpy float64 oracle)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def workload_config(args, N, D):
    from paper_2106_02682_gb300 import synth
    w = synth.WORKLOADS[args.workload]
    return {"workload": args.workload, "lattice": list(w["lattice"]), "cluster": list(w["cluster"]),
            "model": w["kind"], "h": w["h"], "J": 1.0, "clusters": N, "wavevectors": N,
            "pair_dim": D, "precision": args.precision, "mu": 10.0, "nu": 10.0, "eps": 2.0,
            "l2": "flushed (512 MB write) before every timed step", "parallelism": "replicas"}


# ------------------------------------------------------------------ our arm
def run_ours(args):
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_02682_gb300 import synth, ve
    w = synth.WORKLOADS[args.workload]
    dim = len(w["lattice"])
    ham = ve.ve_ham_tfim(dim, 1.0, w["h"]) if w["kind"] == "tfim" else ve.ve_ham_xxz(dim, 1.0, w["h"])
    prec = {"fp64": ve.VE_PREC_FP64, "mixed": ve.VE_PREC_MIXED, "df64": ve.VE_PREC_DF64}[args.precision]
    stream = torch.cuda.Stream()
    opt = ve.ve_default_options(precision=prec, stream=stream.cuda_stream)
    h = ve.ve_create(w["lattice"], w["cluster"], ham, opt)
    N, m, D = ve.ve_dims(h)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    out = {}
    try:
        # mixed precision in the timed loop: force the float32 phase by a zero tolerance.  The
        # timed sweeps are the production path (one captured-graph launch each); the L2 is
        # flushed before each.
        ve.ve_iterate(h, args.warmup, 0.0)
        ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clocks = ClockSampler(local)
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            ev0[k].record(stream)
            ve.ve_iterate(h, 1, 0.0)
            ev1[k].record(stream)
        torch.cuda.synchronize()
        ck = clocks.stop()
        total_ms = sum(a.elapsed_time(b) for a, b in zip(ev0, ev1))
        value, max_ms = job_rate(total_ms, args.steps, world, device="cuda")
        # per-stage times: a separate pass of sweeps issued stage by stage with CUDA events on
        # the handle's stream (same kernels, no graph), L2 flushed before each sweep
        k_prof = max(3, min(args.steps, 50))
        ve.ve_profile(h, 1)
        for _ in range(k_prof):
            with torch.cuda.stream(stream):
                flush.zero_()
            ve.ve_iterate(h, 1, 0.0)
        torch.cuda.synchronize()
        prof = ve.ve_profile_read(h)
        jac_pair, jac_k = ve.ve_profile_sweeps(h)
        ve.ve_profile(h, 0)
        if world > 1:
            torch.distributed.barrier()
        status = ve.ve_get_status(h)

        # ---- end to end through the public API with host buffers
        sb = ve.ve_state_size(h)
        host = torch.empty(sb // 8, dtype=torch.float64, pin_memory=True).numpy()
        ve.ve_get_state(h, host)
        k_e2e = max(3, min(args.steps, 20))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            ve.ve_set_state(h, host)
            ve.ve_iterate(h, 1, 0.0)
            ve.ve_get_state(h, host)
        e2e_s = time.perf_counter() - t0
        e2e = {"value": k_e2e / e2e_s, "unit": UNIT, "h2d_bytes_per_step": sb,
               "d2h_bytes_per_step": sb + 48,
               "how": "per step: ve_set_state from pinned host, ve_iterate(1 sweep) with status "
                      "read-back, ve_get_state to pinned host; wall clock"}

        # ---- roofline of the dominant kernel, from the live per-stage events
        ncanon = (N // 2 + 1) if dim == 1 else None
        if ncanon is None:
            M0 = w["lattice"][0] // w["cluster"][0]
            M1 = w["lattice"][1] // w["cluster"][1]
            ncanon = sum(1 for k0 in range(M0) for k1 in range(M1)
                         if (k0 * M1 + k1) <= (((-k0) % M0) * M1 + (-k1) % M1))
        npass = prof["fft_forward"][1] // max(1, prof["pair"][1])
        work = stage_work(N, D, npass, ncanon)
        dom = max(prof, key=lambda s: prof[s][0])
        ms_launch = prof[dom][0] / max(1, prof[dom][1])
        wk = work.get(dom, {"flops": 0, "bytes": 0})
        if dom in ("pair", "xproj"):
            peak = FP64_PEAK_TFLOPS if prec == 0 else FP32_PEAK_TFLOPS
            achieved = wk["flops"] / (ms_launch * 1e-3) / 1e12
            roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak,
                    "peak_source": ("nominal FP64 rate of the part (recipe table), not in "
                                    "MEASURED_PEAKS.json" if prec == 0 else
                                    "FP32 SIMT (the pipe float32 and double-float words run on): "
                                    "152 SMs x 128 lanes x 2 flop x 2.07 GHz")}
        else:
            peak = 6789.6
            try:
                with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
                    peak = json.load(fh)["hbm_gbs"]
            except (OSError, ValueError, KeyError):
                pass
            achieved = wk["bytes"] / (ms_launch * 1e-3) / 1e9
            roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
        roof["kernel"] = dom
        if D == 256 and prec == 1:
            roof["note"] = ("stage-level: the float32 projections of this stage run as tensor-core "
                            "products (tcgen05, HBM- and chain-bound block rotations) plus SIMT "
                            "block solves; frac counts the nominal eigensolve flops against the "
                            "FP32 SIMT rate. Per-kernel bounds: profiles/"
                            "launches_tfim1d_L4_N1024_mixed.md")
        roof["ms_per_launch"] = ms_launch
        rec = ncu_record(dom, args.workload, args.precision)
        roof["traffic"] = rec.get("dram_bytes_per_launch") if rec else None
        if rec and "pipe_busy_while_resident" in rec:
            # the achieved fraction counts nominal flops only; the pipe counter shows how busy
            # the unit the kernel is bound by actually is (ncu, same sources)
            roof["ncu_pipe_busy"] = {"pipe": rec["pipe"], "frac": rec["pipe_busy_while_resident"]}
        roof["algorithmic_per_launch"] = wk
        stages = {s: {"ms_per_launch": prof[s][0] / max(1, prof[s][1]), "launches": prof[s][1],
                      "share": prof[s][0] / max(1e-12, sum(v[0] for v in prof.values()))}
                  for s in prof}
        # kernels of one sweep (the captured graph holds the same kernel nodes) x timed sweeps
        launches = int(round(sum(v[1] for v in prof.values()) / k_prof)) * args.steps

        # ---- single-GPU extras (N = 1 only: they would hold the other GPUs idle)
        # ---- a batch of 64 paper-size instances against one-at-a-time handles
        batch = None
        if not args.no_ttb and world == 1:
            batch = batch_rate(ve, synth, "paper", 64, 200, ve.VE_PREC_FP64)

        # ---- time to a certified bound: plain float64 against the faster forms
        ttb = None
        if not args.no_ttb and world == 1:
            # on the benchmark workload itself: plain float64 against double-float and mixed
            ttb = plain_race_to_bound(args.workload, ve, synth, stream, args.ttb_max_iter_headline)
            # on the paper's table instance, with the learned warm start and batches
            ttb["paper_instance"] = time_to_bound(args, ve, synth, stream)

        # ---- the general (not translation-invariant) solver on its 128-spin workload
        general = None
        if not args.no_ttb and world == 1:
            general = general_rate(ve, synth, "lrtfim_N128_L1", 3, 10, stream, flush)
            general["workload"] = "lrtfim_N128_L1"

        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "mixed": "f32, then f32x2 (double-float) refinement",
                      "df64": "f32x2 (double-float, 48-bit significand)"}[args.precision],
            "data": "synthetic (seeded spin Hamiltonian, no dataset)",
            "config": workload_config(args, N, D),
            "e2e": e2e, "gpu_launches": launches * world, "roofline": roof, "stages": stages,
            "clocks": ck, "time_to_bound": ttb, "batch": batch, "general": general,
            "jacobi_sweeps_per_eigensolve": {"pair": jac_pair, "wavevector": jac_k},
            "last_status": {"iter": status.iter, "energy_per_spin": status.energy_per_spin,
                            "feas_err": status.feas_err},
        }
    finally:
        ve.ve_destroy(h)
    if rank == 0 and world == 1:
        rate, n, el, cores = oracle_rate(args.workload, args.cpu_seconds)
        out["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": f"{n} full sweeps of {args.workload} in {el:.1f} s "
                                         "(numpy float64 oracle, one warm-up sweep, batched "
                                         f"projections split over {os.cpu_count()} host "
                                         "threads)"}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# ------------------------------------------------------------------ batches
def _solve_to(ve, h, target, chunk, max_sweeps):
    """Iterate in chunks of `chunk` sweeps, certifying after each, until the certified bound per
    spin is >= target.  Returns (sweeps, last certificate, reached)."""
    cert = None
    while True:
        _, st = ve.ve_iterate(h, chunk, 1e-13)
        cert = ve.ve_bound(h)
        if cert.bound_per_spin >= target or st.iter >= max_sweeps:
            return st.iter, cert, cert.bound_per_spin >= target


def plain_race_to_bound(workload, ve, synth, stream, max_iter, check=100):
    """Time to the certified bound on `workload` from fresh handles: plain float64 runs to the
    residual 1e-6 (the metric's stopping rule) and certifies its bound B; double-float and
    mixed precision then run, certifying every `check` sweeps, until their own certified bound
    is >= B - 1e-6.  Wall clock includes every sweep and every certificate."""
    import torch
    w = synth.WORKLOADS[workload]
    dim = len(w["lattice"])
    ham = ve.ve_ham_tfim(dim, 1.0, w["h"]) if w["kind"] == "tfim" else ve.ve_ham_xxz(dim, 1.0, w["h"])
    out = {"workload": workload, "residual_tol": 1e-6, "bound_slack": 1e-6,
           "check_every_sweeps": check}
    h = ve.ve_create(w["lattice"], w["cluster"], ham,
                     ve.ve_default_options(precision=ve.VE_PREC_FP64, stream=stream.cuda_stream))
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        code, st = ve.ve_iterate(h, max_iter, 1e-6)
        cert = ve.ve_bound(h)
        el = time.perf_counter() - t0
    finally:
        ve.ve_destroy(h)
    B = cert.bound_per_spin
    out["fp64"] = {"seconds": el, "sweeps": st.iter, "converged": code == 0,
                   "residual": st.residual, "bound_per_spin": B,
                   "primal_per_spin": cert.primal_per_spin, "iter_per_s": st.iter / el}
    for name, pcode in (("df64", ve.VE_PREC_DF64), ("mixed", ve.VE_PREC_MIXED)):
        h = ve.ve_create(w["lattice"], w["cluster"], ham,
                         ve.ve_default_options(precision=pcode, stream=stream.cuda_stream))
        try:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            n, c, ok = _solve_to(ve, h, B - 1e-6, check, max_iter)
            el2 = time.perf_counter() - t0
        finally:
            ve.ve_destroy(h)
        out[name] = {"seconds": el2, "sweeps": n, "reached": ok, "bound_per_spin": c.bound_per_spin,
                     "primal_per_spin": c.primal_per_spin, "speedup": el / el2}
    return out


def time_to_bound(args, ve, synth, stream):
    """The plain float64 solver runs to the residual 1e-6 (the metric's stopping rule) and
    certifies its bound B; each faster form then runs from a fresh start, certifying every 50
    sweeps, until its own certified bound is within 1e-6 of B: the same certificate, reached
    faster.  The batched form does this for several held-out fields at once."""
    import torch
    from paper_2106_02682_gb300.warmstart import WarmStart, race_to_bound
    tw_ = synth.WORKLOADS[args.ttb_workload]
    tdim = len(tw_["lattice"])

    def ham(x):
        return ve.ve_ham_tfim(tdim, 1.0, x) if tw_["kind"] == "tfim" else ve.ve_ham_xxz(tdim, 1.0, x)

    def opt(p):
        return ve.ve_default_options(precision=p, stream=stream.cuda_stream)

    out = {"workload": args.ttb_workload, "residual_tol": 1e-6, "bound_slack": 1e-6,
           "check_every_sweeps": 50}
    # plain float64: residual 1e-6, then the certificate
    hh = ve.ve_create(tw_["lattice"], tw_["cluster"], ham(tw_["h"]), opt(ve.VE_PREC_FP64))
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        code, st = ve.ve_iterate(hh, args.ttb_max_iter, 1e-6)
        cert = ve.ve_bound(hh)
        el = time.perf_counter() - t0
    finally:
        ve.ve_destroy(hh)
    B = cert.bound_per_spin
    out["fp64"] = {"seconds": el, "sweeps": st.iter, "converged": code == 0,
                   "residual": st.residual, "bound_per_spin": B,
                   "primal_per_spin": cert.primal_per_spin, "iter_per_s": st.iter / el}
    target = B - 1e-6

    def timed(pcode, warm=None, x=None):
        h = ve.ve_create(tw_["lattice"], tw_["cluster"], ham(x if x is not None else tw_["h"]),
                         opt(pcode))
        try:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if warm is not None:
                warm.apply(h, x if x is not None else tw_["h"])
            n, c, ok = _solve_to(ve, h, target, 50, args.ttb_max_iter)
            el = time.perf_counter() - t0
        finally:
            ve.ve_destroy(h)
        return {"seconds": el, "sweeps": n, "reached": ok, "bound_per_spin": c.bound_per_spin,
                "primal_per_spin": c.primal_per_spin}

    out["df64"] = timed(ve.VE_PREC_DF64)
    out["mixed"] = timed(ve.VE_PREC_MIXED)
    # learned warm start: trained on 24 solves of the same family whose fields avoid the ones
    # evaluated, then a mixed-precision solve from its prediction
    wsf = WarmStart(tw_["lattice"], tw_["cluster"], tw_["kind"], n_components=16)
    try:
        xs = np.linspace(0.2, 2.0, 24) + 0.0371
        t0 = time.perf_counter()
        states, _ = wsf.training_states(xs, tol=1e-7, max_iter=60000)
        t_solves = time.perf_counter() - t0
        t0 = time.perf_counter()
        fit_loss = wsf.fit(xs, states, train_steps=4000)
        t_fit = time.perf_counter() - t0
        out["warm_mixed"] = timed(ve.VE_PREC_MIXED, wsf)
        out["warm_mixed"]["training"] = {"instances": len(xs), "solve_seconds": t_solves,
                                         "fit_seconds": t_fit, "fit_loss": fit_loss,
                                         "pca_explained": wsf.explained}
        # batched: held-out fields, each plain float64 on its own against one mixed-precision
        # batch (cold, then started from the learned prediction), each instance to its own
        # float64 bound
        fields = [float(v) for v in np.linspace(0.35, 1.85, args.ttb_batch)]
        plain, targets = [], []
        for x in fields:
            h = ve.ve_create(tw_["lattice"], tw_["cluster"], ham(x), opt(ve.VE_PREC_FP64))
            try:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                _, st = ve.ve_iterate(h, args.ttb_max_iter, 1e-6)
                targets.append(ve.ve_bound(h).bound_per_spin - 1e-6)
                plain.append({"seconds": time.perf_counter() - t0, "sweeps": st.iter})
            finally:
                ve.ve_destroy(h)

        def batched(warm):
            b = ve.ve_create_batch([(tw_["lattice"], tw_["cluster"], ham(x)) for x in fields],
                                   ve.ve_default_options(precision=ve.VE_PREC_MIXED))
            first = [None] * len(fields)
            try:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                if warm is not None:
                    for i, x in enumerate(fields):
                        warm.apply(ve.ve_batch_handle(b, i), x)
                sweeps = 0
                while True:
                    _, sts = ve.ve_batch_iterate(b, 50, 1e-13)
                    sweeps = max(s_.iter for s_ in sts)
                    certs = ve.ve_batch_bound(b)
                    for i, (c, t) in enumerate(zip(certs, targets)):
                        if first[i] is None and c.bound_per_spin >= t:
                            first[i] = sweeps
                    if all(f is not None for f in first) or sweeps >= args.ttb_max_iter:
                        break
                el = time.perf_counter() - t0
            finally:
                ve.ve_batch_destroy(b)
            return {"seconds": el, "sweeps": sweeps, "reached": all(f is not None for f in first),
                    "sweeps_to_bound": first}

        cold_b = batched(None)
        warm_b = batched(wsf)
        # warm and cold copies raced in one batch: the cold start stays as the fallback
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        race = race_to_bound(tw_["lattice"], tw_["cluster"], tw_["kind"], fields, targets, wsf,
                             chunk=50, max_sweeps=args.ttb_max_iter)
        race_s = time.perf_counter() - t0
        plain_s = sum(p_["seconds"] for p_ in plain)
        out["batch"] = {"instances": len(fields), "fields": fields,
                        "plain_fp64_one_at_a_time": {"seconds": plain_s,
                                                     "sweeps": [p_["sweeps"] for p_ in plain]},
                        "mixed_batched": cold_b, "mixed_batched_warm": warm_b,
                        "mixed_batched_warm_or_cold": {
                            "seconds": race_s, "reached": all(r["sweeps"] is not None for r in race),
                            "sweeps_to_bound": [r["sweeps"] for r in race],
                            "copy": [r["copy"] for r in race]},
                        "speedup_batched": plain_s / cold_b["seconds"],
                        "speedup_batched_warm": plain_s / warm_b["seconds"],
                        "speedup_batched_warm_or_cold": plain_s / race_s}
    finally:
        wsf.close()
    return out


def batch_rate(ve, synth, family, count, sweeps, prec, stream=None):
    """Instance-sweeps per second of a batch (one graph launch per sweep) and of the same
    instances advanced one handle at a time."""
    import torch
    inst = synth.batch_instances(family, count)
    triples = [(d["lattice"], d["cluster"],
                ve.ve_ham_tfim(1, 1.0, d["x"]) if d["kind"] == "tfim" else ve.ve_ham_xxz(1, 1.0, d["x"]))
               for d in inst]
    opt = ve.ve_default_options(precision=prec)
    b = ve.ve_create_batch(triples, opt)
    try:
        ve.ve_batch_iterate(b, 3, 0.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ve.ve_batch_iterate(b, sweeps, 0.0)
        el_b = time.perf_counter() - t0
    finally:
        ve.ve_batch_destroy(b)
    el_s = 0.0
    for tr in triples:
        h = ve.ve_create(*tr, opt)
        try:
            ve.ve_iterate(h, 3, 0.0)
            t0 = time.perf_counter()
            ve.ve_iterate(h, sweeps, 0.0)
            el_s += time.perf_counter() - t0
        finally:
            ve.ve_destroy(h)
    clusters = sum(int(np.prod(d["lattice"])) // int(np.prod(d["cluster"])) for d in inst)
    return {"family": family, "instances": count, "clusters_total": clusters,
            "precision": "mixed" if prec else "fp64", "sweeps": sweeps,
            "batched_instance_sweeps_per_s": count * sweeps / el_b,
            "one_at_a_time_instance_sweeps_per_s": count * sweeps / el_s,
            "speedup": el_s / el_b}


def run_batch(args):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_02682_gb300 import synth, ve
    prec = {"fp64": ve.VE_PREC_FP64, "mixed": ve.VE_PREC_MIXED, "df64": ve.VE_PREC_DF64}[args.precision]
    fam = args.workload.split("_", 1)[1]
    count = 256 if fam == "c4" else 64
    r = batch_rate(ve, synth, fam, count, args.steps, prec)
    print(json.dumps({"metric": METRIC, "value": r["batched_instance_sweeps_per_s"],
                      "unit": "instance-sweeps/s", "n_gpus": 1, "steps": args.steps,
                      "warmup": 3, "higher_is_better": True, "scaling": "weak",
                      "vs_baseline": None, "dtype": {0: "f64", 1: "f32+f32x2", 2: "f32x2"}[prec],
                      "data": "synthetic", "config": {"workload": args.workload, **r},
                      "timing": "wall clock around ve_batch_iterate / ve_iterate, no L2 flush"}),
          flush=True)


PROJ_WORKLOADS = {"proj512_b455": (512, 455)}


def run_projection(args):
    """Kernel-only batched PSD projection: 455 real symmetric 512 x 512 matrices (a 64 x 64
    lattice's worth of 3 x 3 clusters, restated as a projection benchmark), float64 in and out,
    through ve_project_psd_sym_large.  Each step projects the whole batch (0.95 GB of input,
    larger than L2); CUDA events on the launching stream."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_02682_gb300 import synth, ve
    n, count = PROJ_WORKLOADS[args.workload]
    prec = {"fp64": ve.VE_PREC_FP64, "mixed": ve.VE_PREC_MIXED, "df64": ve.VE_PREC_DF64}[args.precision]
    steps, warmup = min(args.steps, 3), min(args.warmup, 1)
    A = synth.symmetric_batch(count, n, seed=20210604)
    x = torch.from_numpy(A).cuda()
    y = torch.empty_like(x)
    ws_bytes = ve.ve_project_psd_large_workspace_size(n, False, prec)
    ws = torch.empty(ws_bytes // 8 + 1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()

    def project():
        ve.ve_project_psd_sym_large(x.data_ptr(), y.data_ptr(), n, count, ws.data_ptr(), ws_bytes,
                                    prec, stream.cuda_stream)

    for _ in range(warmup):
        project()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    clocks = ClockSampler(0)
    for a, b in ev:
        a.record(stream)
        project()
        b.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    value = count * steps / (ms * 1e-3)
    # the oracle's projection (numpy eigh) on a sample of the same matrices
    from oracle import ve_oracle as vo
    sample = 16
    t0, c0 = time.perf_counter(), time.process_time()
    vo.proj_psd(A[:sample])
    el = time.perf_counter() - t0
    cores = round((time.process_time() - c0) / el, 2)
    print(json.dumps({
        "metric": "batched PSD projection of 512 x 512 real symmetric matrices", "value": value,
        "unit": "matrices/s", "n_gpus": 1, "steps": steps, "warmup": warmup,
        "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {0: "f64", 1: "f32", 2: "f32x2"}[prec],
        "data": "synthetic (random symmetric, every 7th with eigenvalues +1/-1/0 repeated)",
        "config": {"workload": args.workload, "n": n, "batch": count,
                   "workspace_bytes": ws_bytes, "l2": "inputs 0.95 GB, larger than L2"},
        "gpu_launches": steps, "clocks": ck,
        "cpu_baseline": {"value": sample / el, "unit": "matrices/s", "cores": cores,
                         "kind": "oracle", "sample": f"{sample} matrices, numpy eigh + clip"}}),
        flush=True)


# ------------------------------------------------------------------ general (Algorithm 5)
def general_oracle(name):
    from oracle import alg5
    from oracle import models as mo
    from paper_2106_02682_gb300 import synth
    w = synth.GENERAL_WORKLOADS[name]
    if w["kind"] == "fermion":
        from oracle import fermions
        blocks = fermions.fermion_blocks(w["nsites"], w["L"], w["U"], long_range=w["long_range"])
        pb = alg5.GeneralProblem(blocks, fermionic=True)
    else:
        terms, L = synth.general_terms(name)
        bonds = [(int(s), int(t), B) for (s, t), B in zip(terms["bond_sites"], terms["bond_ops"])]
        blocks = mo.general_blocks(terms["nspins"], L, terms["onsite"], bonds)
        pb = alg5.GeneralProblem(blocks)
    s5 = alg5.general_setup(blocks)
    return alg5, pb, s5, alg5.initial_state(pb, s5)


def general_create(ve, terms, L, opt):
    """A general handle for spin terms (ve_general_create) or fermion terms
    (ve_general_create_fermions)."""
    if "nsites" in terms:
        return ve.ve_general_create_fermions(terms, L, opt)
    return ve.ve_general_create(terms, L, opt)


def general_oracle_rate(name, seconds):
    alg5, pb, s5, st = general_oracle(name)
    alg5.iterate(pb, s5, st)  # warm-up sweep
    n, t0, c0 = 0, time.perf_counter(), time.process_time()
    while True:
        alg5.iterate(pb, s5, st)
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return n / el, n, el, round((time.process_time() - c0) / el, 2)


def general_rate(ve, synth, name, warmup, steps, stream, flush):
    """Sweeps per second of the general solver on workload `name` (CUDA events on the handle's
    stream around each ve_general_iterate(1), L2 flushed before each), then a profiled pass:
    per-stage times, the X step's Jacobi sweeps, and the roofline of its round kernel."""
    import torch
    terms, L = synth.general_terms(name)
    h = general_create(ve, terms, L, ve.ve_default_options(stream=stream.cuda_stream))
    try:
        N, m, D, K = ve.ve_general_dims(h)
        n = N * D
        ve.ve_general_iterate(h, warmup)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        torch.cuda.synchronize()
        for a, b in ev:
            with torch.cuda.stream(stream):
                flush.zero_()
            a.record(stream)
            ve.ve_general_iterate(h, 1)
            b.record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev)
        k_prof = max(3, min(steps, 20))
        ve.ve_general_profile(h, 1)
        for _ in range(k_prof):
            with torch.cuda.stream(stream):
                flush.zero_()
            ve.ve_general_iterate(h, 1)
        torch.cuda.synchronize()
        pms, pl, jac = ve.ve_general_profile_read(h)
        rms, rounds, first_order = ve.ve_general_profile_rounds(h)
        ve.ve_general_profile(h, 0)
        st = ve.ve_general_get_status(h)
        cert = ve.ve_general_bound(h)
    finally:
        ve.ve_general_destroy(h)
    total = sum(pms)
    stages = {s: {"ms_per_sweep": pms[i] / k_prof, "launches_per_sweep": pl[i] / k_prof,
                  "share": pms[i] / max(1e-12, total)} for i, s in enumerate(ve.GENERAL_STAGES)}
    ms_round = rms / max(1, rounds)
    flops_round = 10.0 * n * n
    achieved = flops_round / (ms_round * 1e-3) / 1e12
    xstep_ms = (pms[2] + pms[3]) / k_prof
    return {
        "value": steps / (ms * 1e-3), "ms_per_step": ms / steps,
        "nspins": terms.get("nspins", terms.get("nsites")),
        "clusters": N, "pair_dim": D, "pairs": K, "x_dim": n,
        "launches_per_sweep": sum(pl) / k_prof, "stages": stages,
        "jacobi_sweeps_per_x_step": jac, "x_steps_first_order": first_order / k_prof,
        "roofline": {"bound": "alu", "kernel": "k_dense_round", "achieved": achieved,
                     "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                     "peak_source": "nominal FP64 rate of the part (recipe table), not in "
                                    "MEASURED_PEAKS.json",
                     "ms_per_launch": ms_round, "traffic": None,
                     "algorithmic_per_launch": {"flops": flops_round, "bytes": 64.0 * n * n,
                                                "note": "10 n^2 flops; 8 n^2 words read+written, "
                                                        "L2-resident"}},
        "x_step_nominal_tflops": 13.0 / 3.0 * n ** 3 / (xstep_ms * 1e-3) / 1e12,
        "last_status": {"iter": st.iter, "energy_per_spin": st.energy_per_spin,
                        "feas_err": st.feas_err, "bound_per_spin": cert.bound_per_spin},
    }


def run_general(args):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_02682_gb300 import synth, ve
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    steps, warmup = min(args.steps, 60), max(3, min(args.warmup, 10))
    clocks = ClockSampler(0)
    g = general_rate(ve, synth, args.workload, warmup, steps, stream, flush)
    ck = clocks.stop()
    # end to end through the public API with host buffers
    terms, L = synth.general_terms(args.workload)
    h = general_create(ve, terms, L, ve.ve_default_options(stream=stream.cuda_stream))
    try:
        ve.ve_general_iterate(h, 3)
        sb = ve.ve_general_state_size(h)
        host = torch.empty(sb // 8, dtype=torch.float64, pin_memory=True).numpy()
        ve.ve_general_get_state(h, host)
        k_e2e = 10
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            ve.ve_general_set_state(h, host)
            ve.ve_general_iterate(h, 1)
            ve.ve_general_get_state(h, host)
        e2e_s = time.perf_counter() - t0
    finally:
        ve.ve_general_destroy(h)
    rate, ns, el, cores = general_oracle_rate(args.workload, args.cpu_seconds)
    w = synth.GENERAL_WORKLOADS[args.workload]
    print(json.dumps({
        "metric": "Algorithm 5 ADMM sweeps/s (general Hamiltonian, dense X step)", "value": g["value"],
        "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": warmup, "ms_per_step": g["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": ("synthetic (spinless-fermion ring of the paper's fermionic section, no dataset)"
                 if w["kind"] == "fermion" else
                 "synthetic (seeded disordered long-range spin chain, no dataset)"),
        "config": {"workload": args.workload, **w, "clusters": g["clusters"], "pairs": g["pairs"],
                   "pair_dim": g["pair_dim"], "x_dim": g["x_dim"], "mu": 10.0, "nu": 10.0,
                   "eps": 2.0, "l2": "flushed (512 MB write) before every timed step",
                   "parallelism": "replicas"},
        "e2e": {"value": k_e2e / e2e_s, "unit": UNIT, "h2d_bytes_per_step": sb,
                "d2h_bytes_per_step": sb + 40,
                "how": "per step: ve_general_set_state from pinned host, ve_general_iterate(1 sweep) "
                       "with status read-back, ve_general_get_state to pinned host; wall clock"},
        "gpu_launches": int(round(g["launches_per_sweep"] * steps)), "roofline": g["roofline"],
        "stages": g["stages"], "jacobi_sweeps_per_x_step": g["jacobi_sweeps_per_x_step"],
        "x_steps_first_order": g["x_steps_first_order"],
        "x_step_nominal_tflops": g["x_step_nominal_tflops"], "clocks": ck,
        "last_status": g["last_status"],
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{ns} full sweeps of {args.workload} in {el:.1f} s "
                                   "(numpy float64 oracle, Algorithm 5, one warm-up sweep)"},
    }), flush=True)


def run_general_reference(args):
    alg5, pb, s5, st = general_oracle(args.workload)
    for _ in range(args.warmup):
        alg5.iterate(pb, s5, st)
    t0, c0 = time.perf_counter(), time.process_time()
    for _ in range(args.steps):
        alg5.iterate(pb, s5, st)
    el = time.perf_counter() - t0
    cores = round((time.process_time() - c0) / el, 2)
    value = args.steps / el
    print(json.dumps({
        "impl": "reference", "metric": "Algorithm 5 ADMM sweeps/s (general Hamiltonian, dense X step)",
        "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} full sweeps of {args.workload} after "
                                   f"{args.warmup} warm-up sweeps (numpy float64 oracle)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    args = parse()
    from paper_2106_02682_gb300 import synth
    general = args.workload in synth.GENERAL_WORKLOADS
    if args.impl == "reference":
        if general:
            if dist_env()[1] == 0:
                run_general_reference(args)
        else:
            run_reference(args)
    elif general:
        run_general(args)
    elif args.workload.startswith("batch_"):
        run_batch(args)
    elif args.workload in PROJ_WORKLOADS:
        run_projection(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
