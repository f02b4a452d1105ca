#!/usr/bin/env python
"""FDAS throughput on the SKA-like workload, one JSON line on stdout.

Workload (paper §3: 600 s at 64 us, 193 acceleration trials; the batch of 256
DM trials with BF16 storage beside FP32 is the mixed-precision batch case):
each step searches a batch of `--batch` synthetic series of 2^23 FP32 samples
(noise plus one accelerated sinusoid each) over z in [-96, 96] step 1 (193
templates), 8192-bin overlap-save segments, 16 harmonics, 6-sigma threshold.
The headline runs with BF16 spectra/templates/planes (FP32 arithmetic); the
plain FP32 path is timed on the same inputs beside it.

Timing: W untimed steps, then K steps bracketed by a barrier and
torch.cuda.synchronize(), CUDA events on the caller's stream; every kernel
group is also timed by the library's own events (fdas_profile_*) on the stream
it runs on.  Inputs (8 GiB per batch) and the 1.6 GB power plane exceed the
129 MB L2, so no explicit flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank searches its own batch (DM trials are
independent: weak scaling, no data-path collective) and rank 0 prints the
aggregate over max-over-ranks time.  `--impl reference` times the FP64 CPU
oracle on a bounded sample of the same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "FDAS DM-trials/s (2^23 samples, 193 z); % HBM peak; BF16 vs FP32 at <=3% err"
UNIT = "DM-trials/s"
N_SAMPLES = 1 << 23
TSAMP = 64e-6
Z_MAX, Z_STEP = 96.0, 1.0
SEG_LEN = 8192
N_HARM = 16
SIGMA = 6.0

# FP32 ALU peak of a GB300: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2.07 GHz
FP32_ALU_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _bf16_peak():
    """Dense BF16 tensor peak in TFLOP/s for a kernel timed inside a long
    step (the sustained figure), and its source."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["bf16_tflops_sustained"]), "measured bf16_tflops_sustained"
    except Exception:
        return 1700.0, "fallback (sustained bf16)"


# ---------------------------------------------------------------------------
# clocks and energy (read-only)
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons, power = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_median": statistics.median(power) if power else None}


class Energy:
    """Total-energy counter through NVML (read-only), in joules."""

    def __init__(self, gpu_index: int):
        self.h = None
        try:
            nv = ctypes.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() != 0:
                return
            h = ctypes.c_void_p()
            if nv.nvmlDeviceGetHandleByIndex_v2(gpu_index, ctypes.byref(h)) != 0:
                return
            self.nv, self.h = nv, h
        except OSError:
            self.h = None

    def read(self):
        if self.h is None:
            return None
        v = ctypes.c_ulonglong(0)
        if self.nv.nvmlDeviceGetTotalEnergyConsumption(self.h, ctypes.byref(v)) != 0:
            return None
        return v.value / 1000.0


# ---------------------------------------------------------------------------
# algorithmic work per trial
# ---------------------------------------------------------------------------
def work_model(info, prec_bytes):
    """Bytes/flops per trial of each kernel group (the roofline numerators)."""
    b_s, b_p = (8, 4) if prec_bytes == 4 else (4, 2)
    n, n_r, n_z, L, H = info.n_samples, info.n_r, info.n_z, info.seg_len, info.n_harm
    gather = sum((j / H) ** 2 for j in range(1, H + 1))
    plane = b_p * n_z * n_r
    return {
        # series read + spectrum write (FFT intermediates stay in L2)
        "spectrum_bytes": 4 * n + b_s * n_r,
        # FFT flop model per (segment, template): 4.25 L log2 L + 9 L
        "correlate_flops": (4.25 * L * math.log2(L) + 9 * L) * info.n_seg * n_z,
        "correlate_bytes": b_s * n_r + plane,
        # direct correlation (tensor cores): 8 real flops per complex tap
        # product, sum over templates of (2 m(z) + 1) taps per bin
        "correlate_tc_flops": 8.0 * n_r * sum(
            2 * (8 + math.ceil(abs(i - info.iz0) * info.z_step / 2.0 - 1e-9)) + 1
            for i in range(n_z)),
        # harmonic gathers: unique cells of stream j are (j/H)^2 of the plane
        "harmonic_bytes": plane * gather,
        # what the harmonic sum must read from memory at least: the plane once
        "harmonic_min_bytes": plane,
        "alg_bytes": 4 * n + 2 * b_s * n_r + plane * (1 + gather),
        # floor of the whole path: series read, spectrum written and read,
        # plane written once and read once
        "min_bytes": 4 * n + 2 * b_s * n_r + 2 * plane,
    }


# ---------------------------------------------------------------------------
# oracle on a bounded sample (CPU baseline and reference arm)
# ---------------------------------------------------------------------------
def oracle_trial_seconds(n_rows=9, r_decim=32):
    """Seconds one 2^23-sample trial takes the FP64 oracle, from a sample:
    spectrum + normalisation in full; the direct-correlation plane for
    `n_rows` of the 193 templates (scaled by 193/n_rows); statistics, harmonic
    sum and threshold over a 193 x (N_r/r_decim) plane (scaled by r_decim)."""
    import numpy as np

    import oracle as O
    import synthetic as S
    x, _ = S.batch_series(0, n=N_SAMPLES)
    g = O.geometry(N_SAMPLES, Z_MAX, Z_STEP, N_HARM)
    bank = O.template_bank(g)
    t0 = time.perf_counter()
    Xn, _ = O.normalise(O.spectrum(x), 2048)
    t_spec = time.perf_counter() - t0
    rows = np.linspace(0, g.n_z - 1, n_rows).round().astype(int)
    sub = O.Bank(g, [bank.taps[i] for i in rows], bank.energy[rows])
    sub_geom = O.geometry(N_SAMPLES, Z_MAX, Z_STEP, N_HARM)
    sub_geom.n_z = len(rows)
    sub_geom.m = g.m[rows]
    sub.geom = sub_geom
    t0 = time.perf_counter()
    O.power_plane(Xn, sub)
    t_rows = time.perf_counter() - t0
    small = np.random.default_rng(0).exponential(size=(g.n_z, g.n_r // r_decim))
    t0 = time.perf_counter()
    mean, std = O.plane_stats(small)
    O.candidates(small, g, mean, std, SIGMA)
    t_hs = time.perf_counter() - t0
    total = t_spec + t_rows * g.n_z / len(rows) + t_hs * r_decim
    sample = (f"1 series 2^23: spectrum in full; plane for {len(rows)}/193 templates "
              f"(x{g.n_z / len(rows):.1f}); harmonic sum+threshold on 1/{r_decim} plane "
              f"(x{r_decim})")
    return total, sample, time.perf_counter()


def cpu_baseline():
    import oracle as O
    t0 = time.perf_counter()
    per_trial, sample, _ = oracle_trial_seconds()
    return {"value": 1.0 / per_trial, "unit": UNIT, "cores": O.threads(), "kind": "oracle",
            "sample": sample, "wall_s": round(time.perf_counter() - t0, 2)}


def bf16_vs_oracle(acc):
    """Detection-strength error of the BF16 search against the FP64 oracle
    (part of the CPU leg, after the GPU timing): for each of the series in
    `acc`, every candidate of the BF16 and of the FP32 search has its S_h
    recomputed by the oracle from the FP64 normalised spectrum (one direct
    correlation per gathered cell); the oracle's decision at each of those
    cells uses T_h = mean x G_h with the mean of the series' FP32 plane."""
    import numpy as np

    import oracle as O
    t0 = time.perf_counter()
    g = O.geometry(N_SAMPLES, Z_MAX, Z_STEP, N_HARM)
    bank = O.template_bank(g)
    G = O.gamma_tail_factors(N_HARM, SIGMA)
    worst, n16, n32, n_ora, common16, common32, guard = 0.0, 0, 0, 0, 0, 0, 0
    for x, c16, c32, mean in zip(acc["series"], acc["bf16"], acc["fp32"], acc["mean"]):
        Xn, _ = O.normalise(O.spectrum(x), 2048)
        k16 = {(int(h), int(z), int(r)): float(pw) for h, z, r, pw in
               zip(c16["harm"], c16["iz"], c16["ir"], c16["power"])}
        k32 = {(int(h), int(z), int(r)) for h, z, r in zip(c32["harm"], c32["iz"], c32["ir"])}
        keys = sorted(set(k16) | k32)
        cells, owners = [], []
        for n, (h, iz, ir) in enumerate(keys):
            for k in range(1, h + 1):
                cells.append(O.harmonic_indices(ir, iz, g.iz0, N_HARM, k * (N_HARM // h)))
                owners.append(n)
        if not keys:
            continue
        cells = np.array(cells)
        pw = O.cell_powers(Xn, bank, cells[:, 0], cells[:, 1])
        s_ora = np.bincount(np.array(owners), weights=pw, minlength=len(keys))
        T = {h: mean * G[int(math.log2(h))] for h in (1, 2, 4, 8, 16)}
        ora = {k for k, sv in zip(keys, s_ora) if sv > T[k[0]]}
        near = {k for k, sv in zip(keys, s_ora) if abs(sv - T[k[0]]) <= 0.03 * T[k[0]]}
        for k, sv in zip(keys, s_ora):
            if k in k16:
                worst = max(worst, abs(k16[k] / sv - 1))
        n16 += len(k16)
        n32 += len(k32)
        n_ora += len(ora)
        common16 += len(ora & set(k16))
        common32 += len(ora & k32)
        guard += len((ora ^ set(k16)) - near)
    return {"series": len(acc["series"]), "max_rel_err_bf16": worst,
            "oracle_candidates": n_ora, "bf16_candidates": n16, "fp32_candidates": n32,
            "bf16_common_with_oracle": common16, "fp32_common_with_oracle": common32,
            "bf16_disagreements_outside_3pct_guard": guard,
            "wall_s": round(time.perf_counter() - t0, 2),
            "note": "S_h of every BF16 and FP32 candidate recomputed by the FP64 oracle at its "
                    "gathered cells; oracle decisions with the FP32 plane's mean (within 1e-6 "
                    "of the oracle's in the parity tests)"}


def run_reference(args, rank):
    if rank != 0:
        return
    import oracle as O
    O.build()
    for _ in range(args.warmup):
        oracle_trial_seconds()
    per, walls = [], []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ts = time.perf_counter()
        s, sample, _ = oracle_trial_seconds()
        walls.append(time.perf_counter() - ts)
        per.append(s)
    wall = time.perf_counter() - t0
    # each step runs one bounded sample of one trial (wall time measured) and
    # extrapolates the trial's time from it; a step therefore stands for
    # wall / extrapolated-trial-time trials
    t_trial = statistics.mean(per)
    t_step = statistics.mean(walls)
    value = 1.0 / t_trial
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * t_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config(args),
        "precision": "fp64 oracle",
        "trials_per_step": t_step / t_trial,
        "trial_seconds_extrapolated": t_trial,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": round(wall, 2),
    }
    print(json.dumps(line), flush=True)


def _config(args):
    """The workload (identical for the GPU arm and the reference arm; what
    each arm processes per step is in its own top-level keys)."""
    return {"workload": f"ska_2^{args.n_log2}_193z_h16",
            "n_samples": N_SAMPLES, "tsamp_s": TSAMP, "z_range": [-Z_MAX, Z_MAX],
            "z_step": Z_STEP, "n_z": 193, "seg_len": SEG_LEN, "n_harm": N_HARM,
            "threshold_sigma": SIGMA,
            "l2": "inputs larger than L2 (8 GiB batch, 1.6-3.2 GB plane per trial); no flush",
            "parallelism": "dm-trial shards per GPU, no collective"}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gpu(args, rank, world, local_rank, dist):
    import numpy as np
    import torch

    import paper_2211_13517_gb300 as pkg
    from paper_2211_13517_gb300 import capi, shard
    import synthetic as S

    pkg.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()

    # this rank's block of the job's DM trials, numbered globally
    t_start, t_stop = shard.trial_block(args.batch * world, rank, world)
    ids = list(range(t_start, t_stop))
    xs, sig_params = S.torch_batch_series(t_stop - t_start, N_SAMPLES, base_seed=1000 + t_start,
                                          device=dev)
    torch.cuda.synchronize()
    peak_hbm, peak_src = _peaks()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(v):
        return shard.max_over_ranks(v, dist, dev)

    def timed_stream(plan, inputs, steps, warmup, stream):
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                plan.search(inputs, capacity=1 << 16, stream=stream)
            barrier()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            for _ in range(steps):
                plan.search(inputs, capacity=1 << 16, stream=stream)
            ev1.record(stream)
        barrier()
        return max_over_ranks(ev0.elapsed_time(ev1))

    def timed(plan, inputs, steps, warmup, profile=False, energy=None, clocks=None):
        for _ in range(warmup):
            plan.search(inputs, trial_ids=ids, capacity=1 << 16)
        if profile:
            plan.profile(True)
        barrier()
        if clocks:
            clocks.start()
        e0 = energy.read() if energy else None
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        nfound = 0
        # the search returns once its results are on the host, so the energy
        # counter read after each call brackets that step
        e_steps, e_prev = [], e0
        for _ in range(steps):
            st, c, nf = plan.search(inputs, trial_ids=ids, capacity=1 << 16)
            nfound += nf
            if energy:
                e_now = energy.read()
                if e_now is not None and e_prev is not None:
                    e_steps.append(e_now - e_prev)
                e_prev = e_now
        ev1.record(stream)
        barrier()
        e1 = energy.read() if energy else None
        ck = clocks.stop() if clocks else None
        ms = max_over_ranks(ev0.elapsed_time(ev1))
        prof = plan.profile() if profile else None
        if profile:
            plan.profile(False)
        joules = None
        if e0 is not None and e1 is not None:
            joules = {"total": e1 - e0, "steps": e_steps}
        return ms, prof, joules, ck, nfound

    out = {}
    energy = Energy(local_rank)
    # --- headline: BF16 storage, device-resident inputs -------------------
    plan = capi.Plan(N_SAMPLES, TSAMP, Z_MAX, Z_STEP, SEG_LEN, N_HARM, precision=capi.FDAS_BF16)
    info = plan.info
    clocks = ClockSampler(local_rank)
    # timed without tracing (tracing serialises the kernel groups on one
    # stream); the per-kernel breakdown comes from one traced step after it
    ms_bf16, _, j_bf16, ck, nf_bf16 = timed(plan, xs, args.steps, args.warmup, False, energy,
                                            clocks)
    _, prof_bf16, _, _, _ = timed(plan, xs, 1, 1, True)
    # --- e2e: the same calls with the series in pinned host memory ----------
    # the series in one page-locked host block (a row per series)
    host_block = torch.empty((len(xs), xs[0].numel()), dtype=xs[0].dtype, pin_memory=True)
    for i, x in enumerate(xs):
        host_block[i].copy_(x)
    hosts = list(host_block.unbind(0))
    # the copy rate of these pinned buffers by themselves (torch copies, no
    # library call): the e2e leg needs about 4 N bytes per series at the
    # device rate, and this rate depends on how the host backs the pages
    host_copy_gbs = pinned_copy_gbs(torch, hosts, torch.empty_like(xs[0]))
    for _ in range(max(1, args.warmup // 2)):
        plan.search(hosts, trial_ids=ids, capacity=1 << 16)
    clocks_e2e = ClockSampler(local_rank)
    barrier()
    clocks_e2e.start()
    step_ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    step_ev[0].record(stream)
    nf_e2e = 0
    for i in range(args.steps):
        _, _, nf = plan.search(hosts, trial_ids=ids, capacity=1 << 16)
        nf_e2e += nf
        step_ev[i + 1].record(stream)
    barrier()
    ck_e2e = clocks_e2e.stop()
    ms_e2e = max_over_ranks(step_ev[0].elapsed_time(step_ev[-1]))
    e2e_steps = [round(step_ev[i].elapsed_time(step_ev[i + 1]), 2) for i in range(args.steps)]
    del hosts, host_block
    plan.close()
    # --- FP32 path on the same inputs ---------------------------------------
    ms_fp32 = prof_fp32 = None
    acc_in = None
    if not args.no_fp32:
        plan32 = capi.Plan(N_SAMPLES, TSAMP, Z_MAX, Z_STEP, SEG_LEN, N_HARM,
                           precision=capi.FDAS_FP32)
        ms_fp32, _, j_fp32, _, _ = timed(plan32, xs, args.steps, args.warmup, False, energy)
        _, prof_fp32, _, _, _ = timed(plan32, xs, 1, 1, True)
        # BF16 against FP32 on the first 8 series (untimed): the largest
        # relative error of S over the candidates both report, and how far
        # the two candidate lists agree
        nb = min(8, len(xs))
        _, c32, _ = plan32.search(xs[:nb], trial_ids=ids[:nb], capacity=1 << 18)
        planb = capi.Plan(N_SAMPLES, TSAMP, Z_MAX, Z_STEP, SEG_LEN, N_HARM,
                          precision=capi.FDAS_BF16)
        _, c16, _ = planb.search(xs[:nb], trial_ids=ids[:nb], capacity=1 << 18)
        planb.close()
        # per series: the FP32 plane's mean (for the oracle's thresholds in the
        # CPU leg) and each path's candidates
        means = []
        for x in xs[:nb]:
            spec = plan32.spectrum(x)
            _, pst = plan32.power_plane(spec)
            means.append(float(pst[0]))
            del spec, pst
        plan32.close()
        acc_in = {"series": [x.cpu().numpy() for x in xs[:nb]], "mean": means,
                  "bf16": [c16[c16["trial_id"] == ids[i]] for i in range(nb)],
                  "fp32": [c32[c32["trial_id"] == ids[i]] for i in range(nb)]}
        k32 = {(int(t), int(h), int(z), int(r)): float(pw) for t, h, z, r, pw in
               zip(c32["trial_id"], c32["harm"], c32["iz"], c32["ir"], c32["power"])}
        k16 = {(int(t), int(h), int(z), int(r)): float(pw) for t, h, z, r, pw in
               zip(c16["trial_id"], c16["harm"], c16["iz"], c16["ir"], c16["power"])}
        common = set(k32) & set(k16)
        cmp16 = {"series": nb, "fp32_candidates": len(k32), "bf16_candidates": len(k16),
                 "common": len(common),
                 "max_rel_err_common": max((abs(k16[k] / k32[k] - 1) for k in common),
                                           default=None),
                 "note": "S_h of BF16 storage against FP32 storage on the same series; "
                         "candidates present in one list only lie near the threshold"}
        # FP32 storage with the split (BF16 hi + lo) tensor-core correlation
        plan3 = capi.Plan(N_SAMPLES, TSAMP, Z_MAX, Z_STEP, SEG_LEN, N_HARM,
                          precision=capi.FDAS_FP32, correlator=capi.FDAS_CORR_TENSOR_SPLIT)
        ms_fp32s, _, _, _, nf_fp32s = timed(plan3, xs, args.steps, args.warmup, False)
        _, prof_fp32s, _, _, _ = timed(plan3, xs, 1, 1, True)
        plan3.close()

    # --- fundamental-indexed harmonic sum (FDAS_HARM_FUNDAMENTAL), BF16 ----
    fund = None
    if not args.no_fund:
        planf = capi.Plan(N_SAMPLES, TSAMP, Z_MAX, Z_STEP, SEG_LEN, N_HARM,
                          precision=capi.FDAS_BF16, harmonic_mode=capi.FDAS_HARM_FUNDAMENTAL)
        ms_f, _, _, _, nf_f = timed(planf, xs, args.steps, args.warmup, False)
        _, prof_f, _, _, _ = timed(planf, xs, 1, 1, True)
        planf.close()
        fund = {"value": args.batch * args.steps * world / (ms_f / 1000.0), "unit": UNIT,
                "ms_per_step": ms_f / args.steps,
                "harmonic_ms_per_trial": prof_f["harmonic"][2] / max(1, prof_f["trials"]),
                "candidates_per_trial": nf_f / (args.batch * args.steps),
                "note": "same search with the fundamental-indexed harmonic sum (another "
                        "candidate definition; the headline uses top-harmonic indexing)"}

    # --- interbinning (half-bin plane, 2 N_r columns), BF16, 64 series ----
    ib = None
    if not args.no_interbin:
        nb = min(64, len(xs))
        plani = capi.Plan(N_SAMPLES, TSAMP, Z_MAX, Z_STEP, SEG_LEN, N_HARM,
                          precision=capi.FDAS_BF16, interbin=True)
        ids_keep = ids
        ids = ids[:nb]
        ms_i, _, _, _, nf_i = timed(plani, xs[:nb], args.steps, args.warmup, False)
        _, prof_i, _, _, _ = timed(plani, xs[:nb], 1, 1, True)
        ids = ids_keep
        plani.close()
        ib = {"value": nb * args.steps * world / (ms_i / 1000.0), "unit": UNIT,
              "series_per_step": nb, "ms_per_step": ms_i / args.steps,
              "kernels_ms_per_trial": {g: prof_i[g][2] / max(1, prof_i["trials"])
                                       for g in ("spectrum", "correlate", "harmonic")},
              "candidates_per_trial": nf_i / (nb * args.steps),
              "note": "same search on the half-bin plane (interbinning: |F(r)|^2 and "
                      "(pi/4)^2 |F(r) - F(r+1)|^2 written by the tensor-core epilogue; 2x the "
                      "plane cells)"}

    # --- refinement (Fourier-interpolated power, gradient ascent), FP32 ------
    ref_leg = None
    if not args.no_refine:
        ref_leg = run_refine(args, dev, capi, xs[0], sig_params[0])

    # --- dedispersion upstream of the search: filterbank -> DM-trial series --
    dd = None
    if not args.no_dedisp:
        dd = run_dedisp(args, dev, capi, world)

    # --- uneven batch: full-length and decimated series in one call, graph ---
    uneven = None
    if not args.no_uneven:
        uneven = run_uneven(args, dev, capi, S, timed_uneven=timed_stream)
    trials = args.batch * args.steps * world
    value = shard.weak_scaling_throughput(args.batch * args.steps, world, ms_bf16)
    if rank != 0:
        return
    wm = work_model(info, 2)
    groups = capi.PROFILE_GROUPS

    def group_stats(prof, wmod, tensor=False):
        res = {}
        for g in groups:
            launches, timed_n, ms = prof[g]
            res[g] = {"launches": launches, "timed": timed_n, "ms_total": ms,
                      "ms_per_trial": ms / max(1, prof["trials"])}
        t_sp = res["spectrum"]["ms_per_trial"] / 1e3
        t_co = res["correlate"]["ms_per_trial"] / 1e3
        t_hs = res["harmonic"]["ms_per_trial"] / 1e3
        res["spectrum"]["gbs"] = wmod["spectrum_bytes"] / t_sp / 1e9 if t_sp else None
        flops = wmod["correlate_tc_flops"] if tensor else wmod["correlate_flops"]
        res["correlate"]["tflops"] = flops / t_co / 1e12 if t_co else None
        res["correlate"]["gbs"] = wmod["correlate_bytes"] / t_co / 1e9 if t_co else None
        res["harmonic"]["gbs"] = wmod["harmonic_bytes"] / t_hs / 1e9 if t_hs else None
        return res

    tensor = info.correlator == capi.FDAS_CORR_TENSOR
    k_bf16 = group_stats(prof_bf16, wm, tensor)
    peak_tc, peak_tc_src = _bf16_peak()

    l2_gbs = l2_copy_gbs(torch, dev)

    def roof_of(group):
        traffic = _ncu_traffic(group, "bf16")
        if group == "harmonic":
            t_hs = k_bf16["harmonic"]["ms_per_trial"] / 1e3
            ach = wm["harmonic_min_bytes"] / t_hs / 1e9
            return {"kernel": "harmonic_dedup_kernel<BF16,16>", "bound": "hbm",
                    "achieved": ach, "peak": peak_hbm, "unit": "GB/s",
                    "frac": ach / peak_hbm, "traffic": traffic,
                    "peak_source": f"{peak_src} hbm_gbs (MEASURED_PEAKS.json)",
                    "work": "the plane read once (1.62 GB BF16 per trial), the least the "
                            "harmonic sum must read from HBM",
                    "gathers": {"bytes_per_trial": wm["harmonic_bytes"],
                                "achieved_gbs": k_bf16["harmonic"]["gbs"],
                                "l2_copy_gbs": l2_gbs,
                                "frac_of_l2_copy": k_bf16["harmonic"]["gbs"] / l2_gbs,
                                "note": "plane x sum_j (j/H)^2 = 5.84 planes of gathered BF16 "
                                        "cells, most served from L2; l2_copy_gbs is a torch copy "
                                        "of an L2-resident 32 MiB buffer (read + write bytes)"}}
        a = k_bf16["correlate"]["tflops"]
        if tensor:
            return {"kernel": "correlate_tc_kernel<BF16> (tcgen05)", "bound": "tensor",
                    "achieved": a, "peak": peak_tc, "unit": "TFLOP/s", "frac": a / peak_tc,
                    "traffic": traffic, "peak_source": f"{peak_tc_src} (MEASURED_PEAKS.json)",
                    "work": "8 flops x N_r x sum_z (2 m(z) + 1) per trial (useful taps only)",
                    "plane_write_gbs": k_bf16["correlate"]["gbs"],
                    "plane_write_frac": k_bf16["correlate"]["gbs"] / peak_hbm}
        return {"kernel": "correlate8k_kernel<BF16> (FFT)", "bound": "alu", "achieved": a,
                "peak": FP32_ALU_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": a / FP32_ALU_PEAK_TFLOPS,
                "traffic": traffic,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"}

    # dominant kernel by summed event time
    dom = max(("correlate", "harmonic"), key=lambda g: k_bf16[g]["ms_total"])
    roof = roof_of(dom)
    other = roof_of("harmonic" if dom == "correlate" else "correlate")
    alg_gbs = wm["alg_bytes"] * args.batch * args.steps / (ms_bf16 / 1000.0) / 1e9
    min_gbs = wm["min_bytes"] * args.batch * args.steps / (ms_bf16 / 1000.0) / 1e9
    t_trial = ms_bf16 / 1000.0 / (args.batch * args.steps)
    ncu_bytes = None
    tc, th = _ncu_traffic("correlate", "bf16"), _ncu_traffic("harmonic", "bf16")
    if tc is not None and th is not None:
        ncu_bytes = tc + th + wm["spectrum_bytes"]

    def jstats(j, trials_per_step):
        if not j or not j["steps"]:
            return None
        per = sorted(x / trials_per_step for x in j["steps"])
        return {"median": statistics.median(per), "min": per[0], "max": per[-1],
                "n_steps": len(per), "total_j": j["total"],
                "note": "NVML total-energy counter, read after each step (blocking calls)"}
    # launches of one traced step (the same sequence as an untraced one)
    launches = sum(prof_bf16[g][0] for g in groups) * args.steps
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_bf16 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "storage": "bf16",
        "data": "synthetic", "config": _config(args),
        "precision": "bf16 storage, fp32 arithmetic",
        "series_per_step": args.batch,
        "roofline": roof,
        "roofline_other": other,
        "hbm_alg": {"bytes_per_trial": wm["alg_bytes"], "achieved_gbs": alg_gbs,
                    "peak_gbs": peak_hbm, "frac": alg_gbs / peak_hbm,
                    "note": f"B_alg (5.84 plane-equivalents of harmonic gathers, mostly L2 "
                            f"hits) of the whole path / step time, {peak_src} peak"},
        "hbm_min": {"bytes_per_trial": wm["min_bytes"], "achieved_gbs": min_gbs,
                    "frac": min_gbs / peak_hbm,
                    "note": "B_min: series read, spectrum written + read, plane written once "
                            "and read once, over the step time"},
        "hbm_ncu": ({"bytes_per_trial": ncu_bytes, "achieved_gbs": ncu_bytes / t_trial / 1e9,
                     "frac": ncu_bytes / t_trial / 1e9 / peak_hbm,
                     "note": "DRAM read + write bytes of the correlation and harmonic kernels "
                             "(ncu, profiles/ncu_traffic.json) + the spectrum's, over the "
                             "step time"} if ncu_bytes else None),
        "kernels": k_bf16,
        "e2e": {"value": trials / (ms_e2e / 1000.0), "unit": UNIT,
                "h2d_bytes_per_step": 4 * N_SAMPLES * args.batch,
                "d2h_bytes_per_step": 20 * (nf_e2e // max(1, args.steps)) + 16,
                "step_ms": e2e_steps, "clocks": ck_e2e},
        "e2e_ms_per_step": ms_e2e / args.steps,
        "e2e_h2d_gbs": 4 * N_SAMPLES * args.batch / (ms_e2e / args.steps / 1000.0) / 1e9,
        "e2e_over_value": (trials / (ms_e2e / 1000.0)) / value,
        "e2e_host_copy_gbs": host_copy_gbs,
        "gpu_launches": launches,
        "clocks": ck,
        "joules_per_trial": jstats(j_bf16, args.batch),
        "candidates_per_trial": nf_bf16 / (args.batch * args.steps),
    }
    if ms_fp32 is not None:
        v32 = trials / (ms_fp32 / 1000.0)
        wm32 = work_model(info, 4)
        line["fp32"] = {"value": v32, "ms_per_step": ms_fp32 / args.steps,
                        "kernels": group_stats(prof_fp32, wm32, False),
                        "joules_per_trial": jstats(j_fp32, args.batch),
                        "hbm_alg_frac": wm32["alg_bytes"] * args.batch * args.steps
                        / (ms_fp32 / 1000.0) / 1e9 / peak_hbm}
        line["bf16_speedup_vs_fp32"] = value / v32
        line["bf16_vs_fp32"] = cmp16
        line["fp32_tensor_split"] = {
            "value": args.batch * args.steps * world / (ms_fp32s / 1000.0), "unit": UNIT,
            "ms_per_step": ms_fp32s / args.steps,
            "kernels_ms_per_trial": {g: prof_fp32s[g][2] / max(1, prof_fp32s["trials"])
                                     for g in ("spectrum", "correlate", "harmonic")},
            "note": "FP32 storage, correlation on the tensor cores with BF16 hi + lo operands "
                    "(three products per term, FP32 accumulation; FDAS_CORR_TENSOR_SPLIT)"}
    if uneven is not None:
        line["uneven_batch"] = uneven
    if fund is not None:
        line["fundamental_harmonic"] = fund
    if ib is not None:
        line["interbin"] = ib
    if dd is not None:
        line["dedispersion"] = dd
    if ref_leg is not None:
        line["refine"] = ref_leg
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
        if acc_in is not None:
            line["bf16_vs_oracle"] = bf16_vs_oracle(acc_in)
    print(json.dumps(line), flush=True)


# dedispersion workload: 1024 channels of 0.25 MHz below 1670 MHz, 64 us
# samples, 2^23 output samples per DM trial (the search's series length),
# 128 DM trials from 0 in steps of 0.25 pc cm^-3
DD_CHAN, DD_FTOP, DD_DF, DD_NDM, DD_DMSTEP = 1024, 1670.0, 0.25, 128, 0.25
# shared memory delivers one 4-byte word per lane per clock per SM: 32 words
# x 152 SMs x 2.07 GHz, the bound of a sum that reads every term from it
SMEM_WORDS_PEAK_T = 32 * 152 * 2.07e9 / 1e12


def run_refine(args, dev, capi, x, params):
    """fdas_fourier_power (P and its gradient at arbitrary (r, z)) and
    fdas_refine (50 ascent steps per seed) on one series' FP32 spectrum."""
    import numpy as np
    import torch
    plan = capi.Plan(N_SAMPLES, TSAMP, Z_MAX, Z_STEP, SEG_LEN, N_HARM, precision=capi.FDAS_FP32)
    spec = plan.spectrum(x)
    X = torch.view_as_complex(spec.view(-1, 2))
    n_r = N_SAMPLES // 2
    rng = np.random.default_rng(3)
    n_pts = 8192
    rz = np.stack([rng.uniform(0.01 * n_r, 0.95 * n_r, n_pts), rng.uniform(-90.0, 90.0, n_pts)], 1)
    rz_d = torch.from_numpy(rz).to(dev)
    # work: Y(u) = sum_e X_e exp(2 pi i e u) at 512 nodes over 2m + 1 bins,
    # m = 32 + ceil(|z|/2): 8 flops per complex multiply-add
    m = 32 + np.ceil(np.abs(rz[:, 1]) / 2.0 - 1e-12)
    flops = float(np.sum(8.0 * 512 * (2 * m + 1)))
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        plan.fourier_power(X, rz_d)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        plan.fourier_power(X, rz_d)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    # refinement: 1024 seeds scattered around the injected signal
    r0, z0 = params
    seeds = np.zeros(1024, dtype=capi.SEED_DTYPE)
    seeds["r"] = r0 + rng.uniform(-0.5, 0.5, 1024)
    seeds["z"] = z0 + rng.uniform(-2.0, 2.0, 1024)
    plan.refine(X, seeds[:64], n_steps=50)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = plan.refine(X, seeds, n_steps=50)
    ms_ref = (time.perf_counter() - t0) * 1e3
    # P at the injected parameters, against the peak the seeds reached
    p_inj, _ = plan.fourier_power(X, torch.tensor([[r0, z0]], dtype=torch.float64, device=dev))
    p_inj = float(p_inj.cpu()[0])
    plan.close()
    r_pk, z_pk = float(np.median(out["r"])), float(np.median(out["z"]))
    common = (np.abs(out["r"] - r_pk) < 0.01) & (np.abs(out["z"] - z_pk) < 0.05)
    ach = flops / (ms / 1000.0) / 1e12
    return {"fourier_power": {"points_per_s": n_pts / (ms / 1000.0), "ms_per_launch": ms,
                              "points": n_pts,
                              "roofline": {"bound": "alu", "achieved": ach,
                                           "peak": FP32_ALU_PEAK_TFLOPS, "unit": "TFLOP/s",
                                           "frac": ach / FP32_ALU_PEAK_TFLOPS}},
            "refine": {"seeds_per_s": 1024 / (ms_ref / 1000.0), "ms": ms_ref, "seeds": 1024,
                       "n_steps": 50,
                       "median_accepted_steps": float(np.median(out["steps"])),
                       "reached_common_peak": float(np.mean(common)),
                       "peak_minus_injected": {"dr": r_pk - r0, "dz": z_pk - z0},
                       "power_at_peak": float(np.median(out["power"])),
                       "power_at_injected": p_inj},
            "note": "FP32 spectrum of series 0; P and dP/dr, dP/dz at uniform random (r, z); "
                    "refine times the blocking call (host copies included); its seeds lie within "
                    "0.5 bin and 2 z of the injected (r0, z0) and climb to the one local maximum "
                    "of P there (reached_common_peak: within 0.01 bin and 0.05 z of the seeds' "
                    "median end point), which the series' noise moves from (r0, z0)"}


def run_dedisp(args, dev, capi, world):
    """Incoherent dedispersion of a synthetic N(0,1) filterbank into DM-trial
    series: DM-trials/s and additions/s against the shared-memory bound."""
    import torch
    n_out = N_SAMPLES
    probe = capi.DedispPlan(DD_CHAN, n_out + 1, DD_FTOP, DD_DF, TSAMP, 0.0, DD_DMSTEP, DD_NDM,
                            n_out)
    n_t = n_out + probe.info.max_delay
    probe.close()
    plan = capi.DedispPlan(DD_CHAN, n_t, DD_FTOP, DD_DF, TSAMP, 0.0, DD_DMSTEP, DD_NDM, n_out)
    g = torch.Generator(device=dev)
    g.manual_seed(77)
    fb = torch.randn(DD_CHAN, n_t, generator=g, device=dev, dtype=torch.float32)
    out = torch.empty(DD_NDM, n_out, device=dev, dtype=torch.float32)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        plan.dedisperse(fb, out)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        plan.dedisperse(fb, out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    adds = DD_CHAN * DD_NDM * n_out
    res = {"value": DD_NDM * world / (ms / 1000.0), "unit": "DM-trials/s",
           "ms_per_launch": ms, "n_chan": DD_CHAN, "n_dm": DD_NDM, "n_out": n_out,
           "tile_span": plan.info.tile_span, "max_delay": plan.info.max_delay,
           "roofline": {"bound": "smem", "achieved": adds / (ms / 1000.0) / 1e12,
                        "peak": SMEM_WORDS_PEAK_T, "unit": "T additions/s",
                        "frac": adds / (ms / 1000.0) / 1e12 / SMEM_WORDS_PEAK_T},
           "note": "dedisperse_kernel, inputs larger than L2 (filterbank 34 GB); one 4-byte "
                   "shared-memory word per addition is the bound (less where two DM trials "
                   "share a delay)"}
    # the same trials from an 8-bit filterbank (the usual format; exact sums),
    # then the whole chain: 8-bit filterbank -> DM-trial series -> BF16 search
    del fb
    n_t16 = (n_t + 15) // 16 * 16
    plan.close()
    plan = capi.DedispPlan(DD_CHAN, n_t16, DD_FTOP, DD_DF, TSAMP, 0.0, DD_DMSTEP, DD_NDM, n_out)
    fb8 = torch.randint(0, 256, (DD_CHAN, n_t16), generator=g, device=dev, dtype=torch.uint8)
    for _ in range(args.warmup):
        plan.dedisperse(fb8, out)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        plan.dedisperse(fb8, out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms8 = e0.elapsed_time(e1) / args.steps
    res["u8"] = {"value": DD_NDM * world / (ms8 / 1000.0), "unit": "DM-trials/s",
                 "ms_per_launch": ms8,
                 "frac_of_smem_bound": adds / (ms8 / 1000.0) / 1e12 / SMEM_WORDS_PEAK_T}
    splan = capi.Plan(N_SAMPLES, TSAMP, Z_MAX, Z_STEP, SEG_LEN, N_HARM, precision=capi.FDAS_BF16)
    rows = [out[d] for d in range(DD_NDM)]

    def chain():
        plan.dedisperse(fb8, out)
        return splan.search(rows, capacity=1 << 18)

    for _ in range(max(1, args.warmup // 2)):
        chain()
    torch.cuda.synchronize()
    e0.record(stream)
    n_cand = 0
    for _ in range(args.steps):
        n_cand += chain()[2]
    e1.record(stream)
    torch.cuda.synchronize()
    msc = e0.elapsed_time(e1) / args.steps
    splan.close()
    res["pipeline_u8_to_candidates"] = {
        "value": DD_NDM * world / (msc / 1000.0), "unit": "DM-trials/s", "ms_per_step": msc,
        "candidates_per_trial": n_cand / (args.steps * DD_NDM),
        "note": "8-bit filterbank (1024 channels) -> 128 DM-trial series -> BF16 FDAS search of "
                "all of them, per step"}
    plan.close()
    del fb8, out
    torch.cuda.empty_cache()
    return res


def run_uneven(args, dev, capi, S, timed_uneven):
    """The uneven persistent-batch case: series at full length and decimated
    by 2, 4 and 8 in the proportions 3050 : 959 : 958 : 958, one fdas_search
    per step replayed as one CUDA graph, BF16 storage."""
    import torch
    B = args.uneven_batch
    counts = [round(B * c / 5925) for c in (3050, 959, 958, 958)]
    counts[0] += B - sum(counts)
    xs = []
    for d, c in enumerate(counts):
        if c:
            part, _ = S.torch_batch_series(c, N_SAMPLES >> d, base_seed=5000 + 1000 * d, device=dev)
            xs += part
    torch.cuda.synchronize()
    plan = capi.Plan(N_SAMPLES, TSAMP, Z_MAX, Z_STEP, SEG_LEN, N_HARM, precision=capi.FDAS_BF16,
                     use_graph=True)
    side = torch.cuda.Stream(device=dev)
    steps = max(1, min(args.steps, 3))
    ms = timed_uneven(plan, xs, steps, 1, side)
    plan.close()
    del xs
    torch.cuda.empty_cache()
    equiv = sum(c / (1 << d) for d, c in enumerate(counts))
    return {"series_per_step": B, "split_full_div2_div4_div8": counts,
            "value": B * steps / (ms / 1000.0), "unit": "series/s",
            "full_length_equiv_per_s": equiv * steps / (ms / 1000.0),
            "full_length_equiv_per_step": equiv,
            "steps": steps, "ms_per_step": ms / steps, "use_graph": True, "precision": "bf16",
            "note": "the paper's 5925 DM trials (3050 at full resolution, the rest decimated by "
                    "2, 4 and 8) as one fdas_search call per step, its launches captured and "
                    "replayed as one CUDA graph"}


def pinned_copy_gbs(torch, hosts, dst):
    """Host-to-device rate (GB/s) of one pass of plain copies of the pinned
    host tensors `hosts` into the device tensor `dst` on a side stream."""
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(s):
        for h in hosts:
            dst.copy_(h, non_blocking=True)
    s.synchronize()
    dt = time.perf_counter() - t0
    return sum(h.numel() * h.element_size() for h in hosts) / dt / 1e9


def l2_copy_gbs(torch, dev, mib=32, reps=200):
    """Bytes moved (read + write) per second by torch's copy of an L2-resident
    buffer: a live measure of what L2 delivers to the SMs, beside the HBM
    peak."""
    a = torch.empty(mib << 18, dtype=torch.float32, device=dev).fill_(1.0)
    b = torch.empty_like(a)
    for _ in range(10):
        b.copy_(a)
    st = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        b.copy_(a)
    e1.record(st)
    torch.cuda.synchronize()
    return 2.0 * a.numel() * 4 * reps / (e0.elapsed_time(e1) / 1000.0) / 1e9


def _ncu_traffic(kernel_group, prec):
    """DRAM bytes per launch from the committed ncu summary, if it still
    matches the kernel source; else None."""
    try:
        import hashlib
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            d = json.load(f)
        ent = d[f"{kernel_group}_{prec}"]
        src = os.path.join(ROOT, "paper_2211_13517_gb300", "csrc", ent["source"])
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        return ent["dram_bytes_per_launch_full_size"] if h == ent["source_sha"] else None
    except Exception:
        return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-uneven", action="store_true")
    ap.add_argument("--no-fund", action="store_true",
                    help="skip the fundamental-indexed harmonic-sum leg")
    ap.add_argument("--no-interbin", action="store_true",
                    help="skip the interbinning (half-bin plane) leg")
    ap.add_argument("--no-refine", action="store_true",
                    help="skip the refinement leg")
    ap.add_argument("--no-dedisp", action="store_true",
                    help="skip the dedispersion leg")
    ap.add_argument("--uneven-batch", type=int, default=5925,
                    help="series of the uneven batch (default: the paper's 5925 DM trials)")
    ap.add_argument("--n-log2", type=int, default=23,
                    help="series length 2^n (smaller only for profiling captures)")
    args = ap.parse_args()
    global N_SAMPLES
    N_SAMPLES = 1 << args.n_log2
    if args.warmup < 3 and args.impl == "gb300":
        ap.error("--warmup must be >= 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    dist = None
    if world > 1:
        import torch
        import torch.distributed as td
        torch.cuda.set_device(local_rank)
        td.init_process_group("nccl")
        dist = td
    run_gpu(args, rank, world, local_rank, dist)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
