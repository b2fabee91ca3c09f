#!/usr/bin/env python
"""Throughput of the FVPM photon-transport hot path on GB300.

One step = one hydro step of the radiation solver on a fixed synthetic particle set:
rt_neighbours (cell list, h, pair lists, geometry, source weights) + rt_subcycle
(n_sub x [injection, gradients, pair fluxes + update + grey sink]) + rt_energy.

Metric: pair-group interactions per second, R = P * G * n_sub / t_step, with P the
unordered interacting pairs (r < max(H_i, H_j)) and G the photon groups.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload poisson-sine-beam] [--impl reference]

Under torchrun (N > 1) every rank runs an independent replica (weak scaling); the time
is the max over ranks and the value sums all ranks' units.  --gpus must equal the number of
ranks.  --decompose splits one particle set over the ranks instead (spatial domain
decomposition with halo exchanges; strong scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RT pair interactions/s/group, FP32 vs FP64 at rel err<=1e-5; % of HBM peak"
BREAKDOWN_STEPS = 2     # untimed steps with every kernel bracketed, after the timed ones
PAIR_EVENT_EVERY = 10   # timed steps: events around one pair-pass launch in this many
UNIT = "pair-group interactions/s"
H_OVER_h = 1.825742

# Floating-point operations per pair evaluation, counted on the oracle's own pair arithmetic
# (oracle.Oracle.pair_flops: add, subtract, multiply, divide and square root one each; the
# periodic wrap, comparisons and conversions not counted) over the pairs of these workloads.
# tests/test_flop_counts.py recomputes them with the oracle's counter.  Geometry terms are
# per unordered pair (flux) or per directed neighbour entry (gradient), averaged over the
# set's pairs; the per-group terms are those of a state in the general branch.
PAIR_FLOPS = {
    "poisson-sine-beam": {"flux_geometry": 76.88, "gradient_geometry": 34.94},
    "lognormal-sources": {"flux_geometry": 76.32, "gradient_geometry": 34.66},
}
FLUX_PER_GROUP = 193        # face states (minmod slopes), two M1 closures, GLF
ACC_PER_GROUP = 8           # the flux added to one particle's sums, subtracted from the other's
GRAD_PER_GROUP = 28         # (Q_j - Q_i) psitilde for four components


def pair_flops(workload_key):
    return PAIR_FLOPS.get(workload_key, PAIR_FLOPS["poisson-sine-beam"])


def flux_flops_per_pair(workload_key, G):
    """pair pass: one evaluation per unordered pair."""
    return pair_flops(workload_key)["flux_geometry"] + FLUX_PER_GROUP * G


def grad_flops_per_pair(workload_key, G):
    """gradient pass: both directed entries of an unordered pair."""
    return 2 * (pair_flops(workload_key)["gradient_geometry"] + GRAD_PER_GROUP * G)


def gather_flops_per_pair(G):
    return ACC_PER_GROUP * G


# Algorithmic bytes per particle (float path): pair pass: position/geometry record 48, U in
# 16G, grad U in 48G, U out 16G, alpha 4; gradient: position/geometry 48, U in 16G, grad U
# out 48G; gather: U in 16G, U out 16G, omega and alpha 8 (the pair slots are this
# design's intermediate, not algorithmic).
def flux_bytes_per_particle(G):
    return 52 + 80 * G


def grad_bytes_per_particle(G):
    return 48 + 64 * G


def gather_bytes_per_particle(G):
    return 8 + 32 * G


def sub_bytes_per_particle(G):
    """gradient pass (44 + 16G + 48G) + flux pass (52 + 80G)."""
    return 96 + 144 * G


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), d.get("sm_max_mhz", 2070.0), "measured"
    return 6800.0, 2070.0, "fallback"


def workload(name):
    from paper_2302_12727_gb300 import workloads as W
    return W.WORKLOADS[name]()


# ---------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [t.strip() for t in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def kernel_source_sha1(csrc):
    """sha1 of rt_transport.cu followed by rt_pair.cuh with // comments and blank lines
    removed: the code the counters were taken on, whatever its comments say."""
    lines = []
    for f in ("rt_transport.cu", "rt_pair.cuh"):
        for line in open(os.path.join(csrc, f)).read().splitlines():
            code = line.split("//", 1)[0].rstrip()
            if code.strip():
                lines.append(code)
    return hashlib.sha1("\n".join(lines).encode()).hexdigest()


def traffic_from_profile():
    """DRAM bytes per launch of the sub-cycle kernels from the committed ncu summary, if it
    was taken on the current source of the kernels (else {})."""
    path = os.path.join(ROOT, "profiles", "k_flux_poisson-sine-64^3-G3.md")
    csrc = os.path.join(ROOT, "paper_2302_12727_gb300", "csrc")
    if not os.path.exists(path):
        return {}
    txt = open(path).read()
    h = re.search(r"source_sha1:\s*([0-9a-f]+)", txt)
    if not h or h.group(1) != kernel_source_sha1(csrc):
        return {}
    out = {}
    for k in ("pair_pass", "gradient", "gather"):
        m = re.search(k + r"_dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
        if m:
            out[k] = float(m.group(1))
    return out


# ---------------------------------------------------------------------------------------
def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(t, ws, device):
    """The slowest rank's time (all ranks get it)."""
    if ws == 1:
        return t
    import torch
    import torch.distributed as dist
    tt = torch.tensor([t], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_value(units_per_rank, ws, t_max):
    """Whole-job throughput of independent replicas: every rank's units over the slowest time."""
    return units_per_rank * ws / t_max


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2302_12727_gb300 import Transport, rt_kernel_times, rt_set_profiling

    ws, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    w = workload(args.workload)
    G, n_sub, n = w.n_groups, w.n_steps, w.n
    prec = args.precision
    T = Transport(w.x, w.m, w.xsrc, n_groups=G, c_red=w.c_red, precision=prec, device=dev, riemann=args.riemann)
    diag = T.diagnostics()
    P = diag["n_pairs"]
    dt = args.cfl * diag["dx_min"] / w.c_red
    alpha = None
    if w.kappa:
        f = T.fields()
        alpha = (w.kappa * torch.as_tensor(w.m, device=dev) * f["omega"]).contiguous()
    if args.photo:
        # photo-ionisation sink per group instead of the grey kappa: H0, He0, He+ densities
        # tracing the density with an ionised fraction varying along x; sigma^N of a 1e5 K
        # blackbody in groups split at the three thresholds (library host helper), scaled so
        # that H0 in group 1 gives alpha = kappa rho
        from paper_2302_12727_gb300 import rt_blackbody_groups
        if G != 3:
            raise SystemExit("--photo needs 3 groups")
        rho = w.m * T.fields()["omega"].cpu().numpy()
        xi = 0.5 * (1 + np.sin(2 * np.pi * w.x[0]))
        n_sp = np.stack([rho * (1 - xi), 0.08 * rho * (1 - xi), 0.08 * rho * xi])
        edges = [13.60 * 1.602176634e-12 / 6.62607015e-27, 24.59 * 1.602176634e-12 / 6.62607015e-27,
                 54.42 * 1.602176634e-12 / 6.62607015e-27, math.inf]
        _, sN, _ = rt_blackbody_groups(1e5, edges)
        T.set_absorbers(n_sp, (w.kappa or 0.1) * sN / sN[0, 0])
        alpha = None
    L = T.luminosities(w.Lsrc)
    U0 = T.state(w.U0)
    U = U0.clone()
    # launch variants: given, or the autotuner's choice for this shape (timed before, and
    # outside, the measured region; cached by shape)
    tune_info = {"source": "library default"}
    if args.tuning:
        T.set_tuning(*(int(v) for v in args.tuning.split(",")))
        tune_info = {"source": "--tuning"}
    elif not args.no_autotune:
        from paper_2302_12727_gb300.autotune import autotune
        tune_info = autotune(T, U0, dt, min(n_sub, 10), L, alpha, repeats=2, subcycles_per_build=n_sub)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)
    # the timed steps bracket one pair-pass launch in PAIR_EVENT_EVERY with events (each
    # event pair serialises the graph around its kernel: bracketing all kernels costs ~5% of
    # a step, all pair passes ~2%); the other kernels' times come from an untimed pass after
    # the timed region
    rt_set_profiling(T.ctx, PAIR_EVENT_EVERY + 1)
    stream = torch.cuda.current_stream(dev)

    # moving particles (--drift V): seeded directions at speed V c; every step searches
    # neighbours at the moved positions, sub-cycles, then applies the drift correction
    # U += grad U . v dt_hydro (dt_hydro = n_sub dt) before the particles move on
    drift_ev = []
    if args.drift > 0:
        rs = np.random.default_rng(12727 + 100 + w.seed_id)
        dirs = rs.standard_normal((3, n))
        dirs /= np.linalg.norm(dirs, axis=0, keepdims=True)
        vnp = args.drift * w.c_red * dirs
        vel = torch.as_tensor(vnp, device=dev)
        dt_h = n_sub * dt
        xs = [torch.as_tensor(np.mod(w.x + k * dt_h * vnp, 1.0), device=dev)
              for k in range(args.warmup + args.steps + BREAKDOWN_STEPS)]
    counter = [0]
    bins_info = None
    if args.bins >= 0:
        # individual time bins from each particle's CFL step: dt_min = cfl min dx / c, bins up
        # to args.bins; one hydro step = 2^B min-steps.  Interactions actually evaluated: per
        # min-step s, the pairs with a starting member (s mod 2^b = 0), times G
        bsel, B = T.set_time_bins(None, dt_min=dt, cfl=args.cfl, max_bin=args.bins)
        bh = bsel.cpu().numpy()
        off, cols = T.pairs()
        off, cols = off.cpu().numpy(), cols.cpu().numpy()
        rows = np.repeat(np.arange(n), np.diff(off))
        up = cols > rows
        bk, bl = bh[rows[up]], bh[cols[up]]
        evals = sum(int(np.count_nonzero(((s_ % (1 << bk)) == 0) | ((s_ % (1 << bl)) == 0)))
                    for s_ in range(1 << B))
        bins_info = {"max_bin": int(B), "min_steps": 1 << B, "pair_evaluations": evals,
                     "histogram": np.bincount(bh, minlength=B + 1).tolist()}

    def step():
        k = counter[0]
        counter[0] += 1
        if args.drift > 0:
            T.rebuild(xs[k])
        else:
            T.rebuild()
        if args.bins >= 0:
            T.set_time_bins(None, dt_min=dt, cfl=args.cfl, max_bin=args.bins)
            T.step_bins(U, L, alpha)
            return T.energy(U)
        T.subcycle(U, n_sub, dt, L, alpha)
        if args.drift > 0:
            d0 = torch.cuda.Event(enable_timing=True)
            d1 = torch.cuda.Event(enable_timing=True)
            d0.record(stream)
            T.drift(U, vel, dt_h)
            d1.record(stream)
            drift_ev.append((d0, d1))
        return T.energy(U)

    for _ in range(args.warmup):
        U.copy_(U0)
        step()
    torch.cuda.synchronize()
    drift_ev.clear()

    kflux_n, kgrad_ms, kgrad_n, kpair_ms, kgath_ms = 0, 0.0, 0, 0.0, 0.0
    times = []
    launches0 = T.diagnostics()["kernel_launches"]
    sampler = ClockSampler(local)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        U.copy_(U0)
        flush.fill_(1.0)           # evict the previous step's working set from L2
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        kt = rt_kernel_times(T.ctx)
        kflux_n += kt["flux"][1]
        kpair_ms += kt["flux"][0]
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if ws > 1:
        dist.barrier()
    clocks = sampler.stop()
    launches = T.diagnostics()["kernel_launches"] - launches0
    # untimed pass with every kernel bracketed: the gradient / gather / injection breakdown
    rt_set_profiling(T.ctx, 1)
    bd_sc = 0
    for _ in range(BREAKDOWN_STEPS):
        U.copy_(U0)
        step()
        torch.cuda.synchronize()
        kt = rt_kernel_times(T.ctx)
        kgath_ms += kt["flux_gather"][0]
        kgrad_ms += kt["gradient"][0]
        kgrad_n += kt["gradient"][1]
        bd_sc += n_sub
    rt_set_profiling(T.ctx, 0)
    # U.copy_ and flush.fill_ are torch's kernels, outside the per-step events
    t_total = max_over_ranks(sum(times) / 1e3, ws, dev)
    units_rank = P * G * n_sub * args.steps
    if bins_info:
        units_rank = bins_info["pair_evaluations"] * G * args.steps
    value = job_value(units_rank, ws, t_total)
    ms_step = t_total / args.steps * 1e3

    out = None
    if rank == 0:
        hbm_gbs, sm_max_mhz, peak_kind = measured_peaks()
        # per sub-cycle: one pair-pass launch and one gather launch per group chunk (G <= 4: one);
        # the pair pass from the timed steps, gather and gradient from the untimed pass
        n_sc = args.steps * n_sub
        chunks = (G + 3) // 4                                          # group chunks per pass
        pair_sc_ms = kpair_ms / kflux_n * chunks if kflux_n else 0.0
        gath_sc_ms = kgath_ms / bd_sc if bd_sc else 0.0
        grad_sc_ms = kgrad_ms / bd_sc if bd_sc else 0.0
        pair_avg_s = kpair_ms / kflux_n / 1e3 if kflux_n else None    # one launch of the pair pass
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        alu_peak = n_sm * 128 * 2 * sm_max_mhz * 1e6 / 1e12   # TFLOP/s: SMs x FP32 lanes x FMA x max clock
        flux_flops = P * flux_flops_per_pair(args.workload, G)
        achieved = flux_flops / pair_avg_s / 1e12 if kflux_n else None
        tune = T.tuning()
        # the committed counters hold for the default float kernels on this workload only
        default_shape = (args.workload == "poisson-sine-beam" and prec == "fp32" and args.riemann == "glf"
                         and (tune["flux_variant"], tune["gather_variant"], tune["gradient_variant"]) == (2, 1, 2))
        prof = traffic_from_profile() if default_shape else {}
        traffic = prof.get("pair_pass")
        pair_kernel = {0: "k_flux", 1: "k_flux_staged", 2: "k_flux_tma"}[tune["flux_variant"]]
        grad_kernel = {0: "k_gradient", 1: "k_gradient_g", 2: "k_gradient_s"}[tune["gradient_variant"]]
        gath_kernel = {0: "k_flux_gather", 1: "k_flux_gather_g"}[tune["gather_variant"]]
        chunk_launch = lambda ms: ms / chunks / 1e3 if ms > 0 else None       # s per launch
        grad_s, gath_s = chunk_launch(grad_sc_ms), chunk_launch(gath_sc_ms)
        grad_flops = P * grad_flops_per_pair(args.workload, G) / chunks
        gath_flops = P * gather_flops_per_pair(G) / chunks

        def entry(bound, kernel, work, t_s, peak, unit, traffic_b, alg_bytes):
            a = work / t_s / 1e12 if t_s else None
            d = {"bound": bound, "kernel": kernel, "achieved": a, "peak": peak, "unit": unit,
                 "frac": a / peak if a else None, "traffic": traffic_b, "avg_launch_ms": t_s * 1e3 if t_s else None,
                 "algorithmic_bytes_per_launch": alg_bytes,
                 "hbm_frac_of_" + peak_kind: alg_bytes / t_s / 1e9 / hbm_gbs if t_s else None,
                 "traffic_over_algorithmic_bytes": traffic_b / alg_bytes if traffic_b else None,
                 # the DRAM bytes the kernel actually moves (ncu, cold cache) over its live time
                 "dram_gbs": traffic_b / t_s / 1e9 if (traffic_b and t_s) else None,
                 "dram_frac_of_" + peak_kind: traffic_b / t_s / 1e9 / hbm_gbs if (traffic_b and t_s) else None}
            d["flops_per_launch" if unit == "TFLOP/s" else "bytes_per_launch"] = work
            return d

        rooflines = {
            "pair_pass": entry("alu", pair_kernel, flux_flops, pair_avg_s, alu_peak, "TFLOP/s", traffic,
                               flux_bytes_per_particle(G) * n),
            "gradient": entry("alu", grad_kernel, grad_flops, grad_s, alu_peak, "TFLOP/s", prof.get("gradient"),
                              grad_bytes_per_particle(G) * n),
            # the gather's arithmetic is 8 G flops per pair: it is a memory pass, measured in bytes
            "gather": entry("hbm", gath_kernel, gather_bytes_per_particle(G) * n, gath_s, hbm_gbs / 1e3, "TB/s",
                            prof.get("gather"), gather_bytes_per_particle(G) * n),
        }
        rooflines["gather"]["flops_per_launch"] = gath_flops
        flop_note = ("flops per launch = P x (flux geometry %.2f + %d G) for the pair pass and 2P x (gradient "
                     "geometry %.2f + %d G) for the gradient, per pair counted on the oracle's pair arithmetic "
                     "(oracle pair_flops, tests/test_flop_counts.py)" % (
                         pair_flops(args.workload)["flux_geometry"], FLUX_PER_GROUP,
                         pair_flops(args.workload)["gradient_geometry"], GRAD_PER_GROUP))
        sub_s = (pair_sc_ms + gath_sc_ms + grad_sc_ms) * n_sub / 1e3     # per step
        out = {
            "metric": METRIC,
            "value": value,
            "unit": UNIT,
            "n_gpus": ws,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": ms_step,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "value_per_group": value / G,
            "dtype": "f32" if prec == "fp32" else "f64",
            "data": "synthetic",
            "config": {"workload": w.name, "particles": n, "groups": G, "sub_cycles": n_sub,
                       "sources": w.n_src, "pairs": P, "dt": dt, "dt_rule": f"{args.cfl} * min dx / c (Eq. rt-cfl)",
                       "precision": "fp32 fluxes/gradients, fp64 h/E_i/B_i/energy" if prec == "fp32" else "fp64",
                       "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{ws}",
                       "tuning": T.tuning(), "tuning_source": tune_info.get("source"),
                       "tuning_ms": tune_info.get("ms"), "riemann": args.riemann,
                       "drift_speed_over_c": args.drift,
                       "sink": "photo-ionisation per group" if args.photo else ("grey" if alpha is not None else "none")},
            "roofline": {"bound": "alu", "kernel": f"{pair_kernel} (pair pass)",
                         "achieved": achieved, "peak": alu_peak,
                         "unit": "TFLOP/s", "frac": (achieved / alu_peak) if achieved else None,
                         "traffic": traffic, "peak_source": f"nominal: {n_sm} SMs (device properties) x 128 FP32 lanes x 2 x {sm_max_mhz:.0f} MHz",
                         "flops_per_launch": flux_flops, "avg_launch_ms": pair_avg_s * 1e3 if pair_avg_s else None,
                         "hbm_frac_of_" + peak_kind: (flux_bytes_per_particle(G) * n / pair_avg_s / 1e9) / hbm_gbs
                         if kflux_n else None,
                         "flop_count": flop_note,
                         "traffic_note": "ncu DRAM read + write of one pair-pass launch (cold cache), from "
                                         "profiles/k_flux_poisson-sine-64^3-G3.md; null unless the kernel "
                                         "sources and the launch variants match that capture"},
            "rooflines": dict(rooflines, note="every sub-cycle kernel; the pair pass from the timed steps' events, "
                                              "gradient and gather from the untimed breakdown steps; gather peak "
                                              "= measured HBM copy bandwidth; traffic from the committed ncu "
                                              "summary while the kernel source matches it"),
            "kernels": {"flux_stage_ms_per_subcycle": pair_sc_ms + gath_sc_ms, "gradient_ms_per_subcycle": grad_sc_ms,
                        "pair_flux_ms_per_subcycle": pair_sc_ms, "gather_ms_per_subcycle": gath_sc_ms,
                        "pair_launches_with_events": kflux_n, "gradient_launches_untimed": kgrad_n,
                        "note": f"pair pass: events around one launch in {PAIR_EVENT_EVERY} (sub-cycles 0, "
                                f"{PAIR_EVENT_EVERY}, ...) of the timed steps; gather and gradient: "
                                f"{BREAKDOWN_STEPS} untimed steps after them with every kernel bracketed"},
            "subcycle_only": {"value": P * G * n_sub / sub_s if sub_s > 0 else None, "unit": UNIT,
                              "note": "gradient + pair pass + gather kernel time only (events around each launch)",
                              "hbm_frac_of_" + peak_kind: sub_bytes_per_particle(G) * n * n_sub / sub_s / 1e9 / hbm_gbs
                              if sub_s > 0 else None},
            "time_bins": (dict(bins_info, uniform_equivalent_value=P * G * bins_info["min_steps"] * args.steps / t_total,
                               note="value counts the pair evaluations of the min-steps; uniform_equivalent_value "
                                    "the P G 2^B a uniform dt_min scheme needs for the same hydro step")
                          if bins_info else None),
            "drift": ({"ms_per_step": sum(a.elapsed_time(b) for a, b in drift_ev) / len(drift_ev),
                       "note": "rt_drift (gradients + correction) per step, CUDA events; the step also "
                               "re-searches neighbours at the moved positions"} if drift_ev else None),
            "gpu_launches": int(launches),
            "clocks": clocks,
            "wall_s_timed": wall,
        }
    # end-to-end through the public API with host buffers
    if not args.no_e2e:
        e2e = run_e2e(args, T, w, dt, alpha, L, dev, flush, P)
        if rank == 0:
            out["e2e"] = e2e
    T.close()
    if rank == 0 and not args.no_fp64_plain:
        out["fp64_plain"] = run_fp64_plain(w, args, dev, out["ms_per_step"], P)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(w, args, P)
    if rank == 0 and ws == 1 and not args.no_secondary and args.workload == "poisson-sine-beam":
        out["secondary"] = {name: run_secondary(name, args, dev, flush, fp64=(name == "lognormal-sources"))
                            for name in ("lognormal-sources", "lognormal-sources-large")}
    if rank == 0 and ws == 1 and not args.no_secondary and args.workload == "poisson-sine-beam":
        out["adjoint"] = run_adjoint(args, dev)
    if ws > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


def run_secondary(name, args, dev, flush, fp64=False, steps=2, warmup=1):
    """The larger workloads of the same path, measured after the main line (not part of its
    value): per step rt_neighbours + rt_subcycle(n_sub) + rt_energy with the FP32 graph path
    and the library's default launch shapes, CUDA events, the L2 flushed between steps; with
    fp64, one step of the plain FP64 path launched step by step for the speed-up."""
    import torch
    from paper_2302_12727_gb300 import Transport
    t0 = time.perf_counter()
    w = workload(name)
    t_gen = time.perf_counter() - t0
    G, n_sub = w.n_groups, w.n_steps
    stream = torch.cuda.current_stream(dev)
    res = {"particles": w.n, "groups": G, "sub_cycles": n_sub, "sources": w.n_src, "input_generation_s": t_gen}
    for prec in (("fp32", "fp64") if fp64 else ("fp32",)):
        T = Transport(w.x, w.m, w.xsrc, n_groups=G, c_red=w.c_red, precision=prec, device=dev)
        d = T.diagnostics()
        P = d["n_pairs"]
        dt = args.cfl * d["dx_min"] / w.c_red
        alpha = None
        if w.kappa:
            alpha = (w.kappa * torch.as_tensor(w.m, device=dev) * T.fields()["omega"]).contiguous()
        L = T.luminosities(w.Lsrc)
        U0 = T.state(w.U0)
        U = U0.clone()
        times = []
        n_st = 1 if prec == "fp64" else steps
        for k in range((0 if prec == "fp64" else warmup) + n_st):
            U.copy_(U0)
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            T.rebuild()
            if prec == "fp64":
                for _ in range(n_sub):
                    T.step(U, dt, L, alpha)
            else:
                T.subcycle(U, n_sub, dt, L, alpha)
            T.energy(U)
            e1.record(stream)
            e1.synchronize()
            if k >= (0 if prec == "fp64" else warmup):
                times.append(e0.elapsed_time(e1))
        ms = sum(times) / len(times)
        res[prec] = {"ms_per_step": ms, "value": P * G * n_sub / (ms / 1e3), "unit": UNIT, "pairs": P,
                     "steps": len(times), "path": "plain per-step FP64 launches" if prec == "fp64" else
                     "FP32 graph-captured sub-cycles"}
        T.close()
        del U, U0
        torch.cuda.empty_cache()
    if fp64:
        res["speedup_of_fp32_graph"] = res["fp64"]["ms_per_step"] / res["fp32"]["ms_per_step"]
    return res


def run_adjoint(args, dev, steps=3, warmup=1):
    """The differentiation workload (jittered 32^3 lattice, 2 groups, 8 sources, 16 sub-cycles,
    a checkpoint every 4): the forward sub-cycles and the library adjoint of the loss "E
    summed over the particles within 0.15 of the box centre" (gradients with respect to the
    initial state and the luminosities), in FP64 and FP32.  Wall-clock with the device
    synchronised on both sides (the adjoint call returns after its last kernel); value counts
    the forward pair-group interactions the backward pass differentiates, per second."""
    import torch
    from paper_2302_12727_gb300 import Transport
    w = workload("lattice-sources")
    G, n_sub, k = w.n_groups, w.n_steps, w.ckpt_every
    d = w.x - 0.5
    d -= np.rint(d)
    wt = np.zeros((G, 4, w.n))
    wt[:, 0, np.sqrt((d ** 2).sum(0)) < 0.15] = 1.0
    res = {"workload": w.name, "particles": w.n, "groups": G, "sub_cycles": n_sub, "sources": w.n_src,
           "checkpoint_every": k}
    for prec in ("fp64", "fp32"):
        T = Transport(w.x, w.m, w.xsrc, n_groups=G, c_red=w.c_red, precision=prec, device=dev)
        dg = T.diagnostics()
        P = dg["n_pairs"]
        dt = args.cfl * dg["dx_min"] / w.c_red
        L = T.luminosities(w.Lsrc)
        U0 = T.state(w.U0)
        lam = T.state(wt)
        fwd, bwd = [], []
        for it in range(warmup + steps):
            U = U0.clone()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            T.subcycle(U, n_sub, dt, L)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            dU0, dL = T.adjoint(U0, n_sub, dt, lam, L, None, k)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            if it >= warmup:
                fwd.append(1e3 * (t1 - t0))
                bwd.append(1e3 * (t2 - t1))
        f_ms, b_ms = sum(fwd) / len(fwd), sum(bwd) / len(bwd)
        res[prec] = {"forward_ms": f_ms, "adjoint_ms": b_ms, "adjoint_over_forward": b_ms / f_ms,
                     "value": P * G * n_sub / (b_ms / 1e3), "unit": UNIT, "pairs": P, "steps": len(bwd),
                     "finite": bool(torch.isfinite(dU0).all().item() and torch.isfinite(dL).all().item())}
        T.close()
    return res


def run_e2e(args, T, w, dt, alpha, L, dev, flush, P):
    """Same steps through the Python API, every step copying the positions and the initial
    state from pinned host memory and the final state and energy back."""
    import torch
    x_h = torch.from_numpy(np.ascontiguousarray(w.x)).pin_memory()
    U_h = torch.from_numpy(np.ascontiguousarray(w.U0).astype(np.float32 if T.precision == "fp32" else np.float64)).pin_memory()
    out_h = torch.empty_like(U_h).pin_memory()
    stream = torch.cuda.current_stream(dev)
    G, n_sub = w.n_groups, w.n_steps
    times = []
    for k in range(args.warmup + args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        xd = x_h.to(dev, non_blocking=True)
        U = U_h.to(dev, non_blocking=True)
        T.rebuild(xd)
        T.subcycle(U, n_sub, dt, L, alpha)
        E = T.energy(U)
        out_h.copy_(U, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        if k >= args.warmup:
            times.append(e0.elapsed_time(e1))
    t = sum(times) / 1e3
    bi = x_h.numel() * 8 + U_h.numel() * U_h.element_size()
    bo = out_h.numel() * out_h.element_size() + 8 * G
    return {"value": P * G * n_sub * len(times) / t, "unit": UNIT, "h2d_bytes_per_step": int(bi),
            "d2h_bytes_per_step": int(bo), "ms_per_step": t / len(times) * 1e3}


def run_fp64_plain(w, args, dev, ms_fp32, P):
    """The plain FP64 path: FP64 kernels launched one step at a time (no graph)."""
    import torch
    from paper_2302_12727_gb300 import Transport
    G, n_sub = w.n_groups, w.n_steps
    T = Transport(w.x, w.m, w.xsrc, n_groups=G, c_red=w.c_red, precision="fp64", device=dev, riemann=args.riemann)
    d = T.diagnostics()
    dt = args.cfl * d["dx_min"] / w.c_red
    alpha = None
    if w.kappa:
        f = T.fields()
        alpha = (w.kappa * torch.as_tensor(w.m, device=dev) * f["omega"]).contiguous()
    L = T.luminosities(w.Lsrc)
    U0 = T.state(w.U0)
    reps = 2
    times = []
    for k in range(reps + 1):
        U = U0.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        T.rebuild()
        for _ in range(n_sub):
            T.step(U, dt, L, alpha)
        T.energy(U)
        torch.cuda.synchronize()
        if k:
            times.append(time.perf_counter() - t0)
    T.close()
    ms = statistics.median(times) * 1e3
    return {"ms_per_step": ms, "value": P * G * n_sub / (ms / 1e3), "unit": UNIT,
            "speedup_of_fp32_graph": ms / ms_fp32}


def oracle_step_times(w, P, n_src_steps=2, riemann="glf"):
    import oracle
    o_t0 = time.perf_counter()
    o = oracle.Oracle(w.x, w.m, w.xsrc, n_groups=w.n_groups, c_red=w.c_red, riemann=riemann)
    t_build = time.perf_counter() - o_t0
    dx = (o.V / (4 * np.pi / 3)) ** (1 / 3)
    dt = 0.9 * dx.min() / w.c_red
    alpha = w.kappa * w.m * o.omega if w.kappa else None
    t0 = time.perf_counter()
    o.run(w.U0, n_src_steps, dt, w.Lsrc, alpha)
    t_step = (time.perf_counter() - t0) / n_src_steps
    return t_build, t_step, oracle.num_threads()


def cpu_baseline(w, args, P):
    t_build, t_step, cores = oracle_step_times(w, P, 2, args.riemann)
    T = t_build + w.n_steps * t_step
    return {"value": P * w.n_groups * w.n_steps / T, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"full {w.n}-particle set: oracle build ({t_build:.2f} s) + 2 of the {w.n_steps} steps "
                      f"({t_step:.2f} s each) timed; the {w.n_steps}-step figure extrapolated from them"}


def run_reference(args):
    """The oracle as it stands on the host cores, on the same workload: its build is timed
    once, then every step is one sampled sub-cycle (injection, gradients, fluxes, update and
    sink over the whole particle set); the value counts the pair-group interactions of the
    timed sub-cycles only."""
    ws, rank, local = dist_setup()
    if rank != 0:
        return
    w = workload(args.workload)
    import oracle
    t0 = time.perf_counter()
    o = oracle.Oracle(w.x, w.m, w.xsrc, n_groups=w.n_groups, c_red=w.c_red, riemann=args.riemann)
    t_build = time.perf_counter() - t0
    off, _ = o.pairs()
    P = int(off[-1]) // 2
    dx = (o.V / (4 * np.pi / 3)) ** (1 / 3)
    dt = args.cfl * dx.min() / w.c_red
    alpha = w.kappa * w.m * o.omega if w.kappa else None
    U = np.array(w.U0, dtype=np.float64)
    times = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        U, _ = o.run(U, 1, dt, w.Lsrc, alpha)
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    cores = oracle.num_threads()
    t_step = sum(times) / len(times)
    val = P * w.n_groups / t_step
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": w.name, "particles": w.n, "groups": w.n_groups, "sub_cycles": w.n_steps,
                      "pairs": P, "riemann": args.riemann, "dt": dt},
           "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"each step is one sub-cycle of the {w.n_steps} of a hydro step on the full "
                                      f"{w.n}-particle set, all {args.steps} timed; the oracle's neighbour build "
                                      f"({t_build:.2f} s, once per hydro step) is timed before them and not "
                                      f"included"},
           "oracle_build_s": t_build,
           "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def run_decomposed(args):
    """One particle set over N ranks (paper_2302_12727_gb300.domain): a step is n_sub
    sub-cycles (ghost exchange + transport step on every rank) and the energy all-reduce; the
    decomposition's build runs once before the timed steps and is not timed."""
    import torch
    import torch.distributed as dist

    from paper_2302_12727_gb300 import domain

    ws, rank, local = dist_setup()
    if args.backend == "gloo":
        # host-staged exchanges; the ranks may share a GPU (a check of this path on one GPU:
        # no kernel of one rank waits on another's)
        local = local % torch.cuda.device_count()
    torch.cuda.set_device(local)
    dist.init_process_group(args.backend)
    dev = torch.device("cuda", local)
    w = workload(args.workload)
    G, n_sub = w.n_groups, w.n_steps
    eng = domain.CudaEngine(G, w.c_red, precision=args.precision, device=dev, riemann=args.riemann)
    D = domain.DistributedTransport(w.x, w.m, w.xsrc, eng, exchange=args.exchange)
    # every particle's row is exact in its owner's context: the owned rows sum to 2P
    rows_owned = float(eng.pair_counts()[:D.plan.n_owned].sum())
    om_own = eng.t.fields()["omega"].cpu().numpy()[:D.plan.n_owned]
    dx_min = D._all_max(-float(((1.0 / om_own) / (4 * np.pi / 3)).min() ** (1 / 3)))
    dt = args.cfl * (-dx_min) / w.c_red
    alpha = None
    if w.kappa:
        om = np.zeros(w.n)
        om[D.plan.owned] = eng.t.fields()["omega"].cpu().numpy()[:D.plan.n_owned]
        alpha = w.kappa * w.m * D._all_sum(om)
    U0 = D.local_state(w.U0)
    L, al = D.local_luminosities(w.Lsrc), D.local_alpha(alpha)
    U = U0.clone()
    for _ in range(args.warmup):
        U.copy_(U0)
        D.subcycle(U, n_sub, dt, L, al)
        D.energy(U)
    torch.cuda.synchronize()
    times = []
    for _ in range(args.steps):
        U.copy_(U0)
        dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        D.subcycle(U, n_sub, dt, L, al)
        D.energy(U)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    t_max = max_over_ranks(sum(times), ws, dev if args.backend == "nccl" else torch.device("cpu"))
    P = int(D._all_sum([rows_owned])[0]) // 2
    held = float(D._all_sum([len(D.plan.local)])[0]) / w.n      # every rank takes part
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": P * G * n_sub * args.steps / t_max, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64",
            "data": "synthetic",
            "config": {"workload": w.name, "particles": w.n, "groups": G, "sub_cycles": n_sub,
                       "parallelism": f"domain decomposition x{ws}", "exchange": args.exchange,
                       "particles_held_over_owned": held, "pairs": P,
                       "note": "host-timed steps (sub-cycles with halo exchanges + energy all-reduce); "
                               "the decomposition's build is not timed"}}))
    D.close()
    dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="poisson-sine-beam",
                    help="lattice-point-source, poisson-sine-beam (the default), lattice-sources, "
                         "lognormal-sources or lognormal-sources-large")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--cfl", type=float, default=0.9)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64-plain", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the secondary measurements (the 2,097,152- and 16,777,216-particle workloads "
                         "and the adjoint on the 32,768-particle differentiation workload)")
    ap.add_argument("--riemann", default="glf", choices=["glf", "hll"],
                    help="pair-flux Riemann solver (Eq. riemann-GLF or Eq. riemann-HLL)")
    ap.add_argument("--tuning", default="", help="flux,gather,gradient variants of the float pair kernels")
    ap.add_argument("--no-autotune", action="store_true", help="keep the library's default launch variants")
    ap.add_argument("--bins", type=int, default=-1,
                    help="individual time bins from the CFL step, up to this bin (one hydro step per step)")
    ap.add_argument("--photo", action="store_true",
                    help="per-group photo-ionisation sink (rt_set_absorbers) instead of the grey kappa")
    ap.add_argument("--drift", type=float, default=0.0,
                    help="move the particles at this fraction of c (drift correction + new neighbours every step)")
    ap.add_argument("--backend", default="nccl", choices=["nccl", "gloo"],
                    help="process-group backend of --decompose (gloo: exchanges through the host)")
    ap.add_argument("--exchange", default="state", choices=["state", "gradients"],
                    help="what --decompose exchanges per sub-cycle: the ghosts' states (deep halo) or "
                         "states and gradients (the thesis's pattern, shallow halo)")
    ap.add_argument("--decompose", action="store_true",
                    help="with N > 1 ranks: one particle set split over the ranks by the spatial domain "
                         "decomposition (halo exchanges over NCCL) instead of N independent replicas")
    args = ap.parse_args()
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if args.gpus != ws:
        raise SystemExit(f"--gpus {args.gpus} but {ws} rank(s): launch N ranks with "
                         f"'python -m torch.distributed.run --nproc-per-node N bench.py --gpus N'")
    if args.impl == "reference":
        run_reference(args)
    elif args.decompose and ws > 1:
        run_decomposed(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
