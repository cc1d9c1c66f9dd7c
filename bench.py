#!/usr/bin/env python3
"""Benchmark: direct dedispersion of the single-beam HTRU-shaped gulp.

Workload (one step): 1024 channels of 0.390625 MHz (1581.8 -> 1181.8 MHz,
highest first), 64 us sampling, 2-bit packed input of 2^19 output samples plus
the maximum delay (20464 samples at DM 999), 1500 trial DMs (step 0.25 over
0-100, 0.5 over 100-300, 1.0 over 300-1000), uint32 output [1500 x 2^19].

Metric: Gsamp/s = nchan * ndm * nsamp_out / step time (whole job over all
ranks).  Every rank dedisperses its own beam's gulps (weak scaling, no
data-path collective); the only collective is the max-over-ranks timing.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

NCHAN = 1024
NOUT = 1 << 19
TSAMP = synth.TSAMP_HTRU
WORKLOAD = "single HTRU-shaped beam: 1024 ch x 1500 DM x 2^19 samples, 2-bit"
METRIC = "dedispersion Gsamp/s (nchan*ndm*nsamp)"
KERNEL_SRCS = [os.path.join(ROOT, "paper_1112_0065_gb300", "csrc", f)
               for f in ("dedisp_kernels.cu", "tiled_tile.cuh", "tiled_launch.cuh", "tiled_g64.cu", "tc.cuh")]
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "dd_tiled_kernel_htru_1024x1500.md")
WIDTHS = tuple(1 << k for k in range(11))
CLF_BATCH = 32768  # snippets per classifier launch (a gulp's candidates in one launch chain)
NCU_NN_BATCH = 8192  # snippets of the classifier's profiling case
# multiply-adds per snippet of the classifier: 3x3 convolutions 1->16 on 64x64,
# 16->32 on 32x32, 32->64 on 16x16, 64->64 on 8x8, then fc 1024->128 and 128->1
CLF_MAC_PER_SNIPPET = (64 * 64 * 16 * 1 + 32 * 32 * 32 * 16 + 16 * 16 * 64 * 32 + 8 * 8 * 64 * 64) * 9 + 1024 * 128 + 128


def kernel_source_hash() -> str:
    """sha256 (first 16 hex digits) of the tiled kernel's sources, in order,
    without their whole-line // comments (a comment edit changes no kernel)."""
    h = hashlib.sha256()
    for path in KERNEL_SRCS:
        with open(path, "rb") as f:
            for line in f:
                if not line.lstrip().startswith(b"//"):
                    h.update(line)
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def alu_peak_tadds(sm_mhz: float, sms: int = 152) -> float:
    """INT32 add peak: 152 SMs x 128 INT32 lanes per SM per clock x SM clock."""
    return sms * 128 * sm_mhz * 1e6 / 1e12


def profiled_traffic(shape):
    """DRAM bytes per launch recorded by the committed ncu summary, if it was
    taken on the current kernel source and on the tile shape the bench runs
    (shape = (DMs per CTA, words per lane, channels per stage)); the summary
    lists one `kernel_shape_dram: D W G bytes` line per profiled shape."""
    if not os.path.exists(PROFILE_SUMMARY):
        return None
    src_hash = kernel_source_hash()
    h = None
    per_shape = {}
    with open(PROFILE_SUMMARY) as f:
        for line in f:
            if line.startswith("kernel_source_sha256_16:"):
                h = line.split(":", 1)[1].strip()
            if line.startswith("kernel_shape_dram:"):
                v = line.split(":", 1)[1].split()
                per_shape[tuple(int(x) for x in v[:3])] = float(v[3])
    return per_shape.get(tuple(shape)) if h == src_hash else None


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

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
                                          "--format=csv,noheader,nounits", "-lms", "100"],
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
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle on the host cores
# ---------------------------------------------------------------------------

_HOST_GULP = {}
CANDS_PER_GULP = 20000  # the GPU pipeline's typical candidate count on this workload (measured, ~20k)


def _host_workload(seed: int = 1):
    import oracle

    f = synth.band_freqs(NCHAN)
    dms_all = synth.dm_list_piecewise(1000.0)
    delays_all = oracle.delay_table(f, TSAMP, dms_all)
    nsamp = NOUT + int(delays_all.max())
    if seed not in _HOST_GULP:
        rng = np.random.default_rng(seed)
        lv = None
        packed = synth.noise_packed(rng, NCHAN, nsamp)
        _HOST_GULP[seed] = packed
        del lv
    return f, dms_all, delays_all, nsamp, _HOST_GULP[seed]


def cpu_oracle_step(ndm_sample: int, nsnip: int = 4, seed: int = 1):
    """Time the oracle on a bounded sample of one step and extrapolate to the
    whole step: ndm_sample of the 1500 DM rows dedispersed over the full gulp
    (OpenMP over rows), the search (running median, boxcars 1..1024) of one
    full row, and the classifier on nsnip snippets; the step time is
    1500 x (dedispersion + search per row) + CANDS_PER_GULP x (classifier per
    snippet)."""
    import oracle

    f, dms_all, delays_all, nsamp, packed = _host_workload(seed)
    idx = np.linspace(0, 1499, ndm_sample).round().astype(int)
    idx[-1] = 1499  # keep the largest delay so the output length is the workload's
    delays = np.ascontiguousarray(delays_all[idx])
    t0 = time.perf_counter()
    out = oracle.dedisperse(delays, packed, nsamp)
    t_dd = time.perf_counter() - t0
    assert out.shape == (ndm_sample, NOUT)
    row = out[ndm_sample // 2][None, :]
    t0 = time.perf_counter()
    y = oracle.baseline(row, 4096)
    best, bw = oracle.best_snr(y, WIDTHS)
    t_search = time.perf_counter() - t0
    rng = np.random.default_rng(seed)
    x = oracle.float_to_bf16_bits(rng.standard_normal((nsnip, 64, 64)).astype(np.float32))
    params = np.zeros(oracle.nn_param_count(), np.float32)
    t0 = time.perf_counter()
    oracle.nn_forward(params, x)
    t_nn = time.perf_counter() - t0
    step_s = 1500 * (t_dd / ndm_sample + t_search) + CANDS_PER_GULP * t_nn / nsnip
    sampled_s = t_dd + t_search + t_nn
    return NCHAN * 1500 * NOUT / step_s / 1e9, step_s, sampled_s, oracle.num_threads()


def cpu_baseline(ndm_sample: int = 64):
    gs, step_s, sampled, thr = cpu_oracle_step(ndm_sample)
    return {"value": round(gs, 5), "unit": "Gsamp/s", "cores": thr, "kind": "oracle",
            "sample": f"{ndm_sample} of 1500 DM rows dedispersed over the full 2^19-sample gulp ({thr} OpenMP "
                      f"threads), the search of 1 full row (1 thread), the classifier on 4 snippets; extrapolated "
                      f"to 1500 rows and {CANDS_PER_GULP} candidates = {step_s:.0f} s per step; {sampled:.1f} s of "
                      f"CPU work sampled"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    n = 32
    for _ in range(args.warmup):
        cpu_oracle_step(n)
    vals, steps_s, sampled = [], [], 0.0
    thr = 1
    for _ in range(args.steps):
        gs, st, sm, thr = cpu_oracle_step(n)
        vals.append(gs)
        steps_s.append(st)
        sampled += sm
    value = float(np.mean(vals)) if vals else 0.0
    cb = {"value": round(value, 5), "unit": "Gsamp/s", "cores": thr, "kind": "oracle",
          "sample": f"per step: {n} of 1500 DM rows dedispersed over the full gulp, the search of 1 row, the "
                    f"classifier on 4 snippets, extrapolated to the whole step ({CANDS_PER_GULP} candidates); "
                    f"{sampled:.1f} s of CPU work sampled in total"}
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": "Gsamp/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * float(np.mean(steps_s)), 1) if steps_s else None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "step": "dedispersion + running-median baseline + boxcar matched "
                       "filter + classifier, the CPU oracle on a sample of the step, extrapolated",
                       "nchan": NCHAN, "ndm": 1500, "nsamp_out": NOUT},
            "cpu_baseline": cb,
            "e2e": {"value": round(value, 5), "unit": "Gsamp/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def beam_gulp(nchan, nsamp, nout, dm_max, seed, offsets_for_dm, dev, npulses=20):
    """Packed gulp of one beam: quantised noise plus the multibeam injection
    recipe (dispersed pulses, 5% stuck channels, zero-DM bursts)."""
    rng = np.random.default_rng(seed)
    rec = synth.draw_recipe(rng, nchan, nout, dm_max, offsets_for_dm, npulses=npulses)
    d = synth.device_noise_packed(nchan, nsamp, seed=seed, device=dev)
    synth.device_apply_recipe(d, nsamp, rec)
    return d


class GulpPipeline:
    """One gulp through the whole hot path: dedispersion, baseline, matched
    filter, grouping, snippets and classifier scores."""

    def __init__(self, P, plan, nout, clf, dev, max_cands=1 << 17):
        import torch

        self.P, self.plan, self.nout, self.clf = P, plan, nout, clf
        self.nsamp = nout + plan.maxdelay
        self.out = plan.alloc_output(self.nsamp, dev)
        self.search = P.Search(plan.ndm, nout, nchan=plan.nchan, half_window=4096, widths=WIDTHS, thresh=6.0,
                               max_cands=max_cands, full_map=False)
        self.snip = torch.empty((max_cands, 64, 64), dtype=torch.bfloat16, device=dev)
        self.logits = torch.empty(max_cands, dtype=torch.float32, device=dev)
        self.max_cands = max_cands
        self.last_n = 0
        self.last_nhot = 0

    def step(self, d_in, ev=None):
        """ev: optional list of 5 CUDA events marking the stage boundaries."""
        import torch

        s = torch.cuda.current_stream()
        if ev:
            ev[0].record(s)
        self.plan.execute(d_in, self.nsamp, self.out)
        if ev:
            ev[1].record(s)
        self.search.run(self.out, self.plan.ndm, self.nout)
        if ev:
            ev[2].record(s)
        res = self.search.result()                                 # host reads the group count
        n = min(res["ngroups"], self.max_cands)
        self.last_nhot = res["nhot"]
        self.search.snippets(n, self.snip)
        if ev:
            ev[3].record(s)
        for i in range(0, n, CLF_BATCH):
            k = min(CLF_BATCH, n - i)
            self.clf.forward(self.snip[i:i + k], out=self.logits[i:i + k])
        if ev:
            ev[4].record(s)
        self.last_n = n
        # kernels launched: dedispersion 1, search 13 (median, thresholds, matched filter, tile scan, runs,
        # row joins, compress, ids, group reduce, marks, count, scan, write), snippets (if any),
        # classifier 7 per chunk (weight image, 4 convolutions, fc1, fc2)
        return 1 + 13 + (1 if n else 0) + 7 * ((n + CLF_BATCH - 1) // CLF_BATCH)

    def baseline_variants(self, reps=3):
        """The search stage on the last gulp's dedispersed rows with the running
        median (default) and with the paper's running mean: time of each."""
        import torch

        P = self.P
        alt = P.Search(self.plan.ndm, self.nout, nchan=self.plan.nchan, half_window=4096, widths=WIDTHS,
                       thresh=6.0, max_cands=self.max_cands, full_map=False, baseline="mean")
        s = torch.cuda.current_stream()
        out = {}
        for name, srch in (("median", self.search), ("mean", alt)):
            srch.run(self.out, self.plan.ndm, self.nout)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(reps):
                srch.run(self.out, self.plan.ndm, self.nout)
            e1.record(s)
            torch.cuda.synchronize()
            out[name + "_search_ms"] = round(e0.elapsed_time(e1) / reps, 3)
            res = srch.result()
            out[name + "_groups"] = res["ngroups"]
            out[name + "_hot_cells"] = res["nhot"]
        alt.close()
        return out

    def classifier_variants(self, reps=3):
        """The last gulp's candidates scored by the fixed-order forward and by
        the tensor-core forward: time of each (CUDA events) and the largest
        logit difference."""
        import torch

        n = self.last_n
        if n == 0:
            return None
        s = torch.cuda.current_stream()
        tc_logits = torch.empty_like(self.logits)
        out = {}
        for name, tc, dst in (("exact", False, self.logits), ("tensor_cores", True, tc_logits)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(reps):
                for i in range(0, n, CLF_BATCH):
                    k = min(CLF_BATCH, n - i)
                    self.clf.forward(self.snip[i:i + k], out=dst[i:i + k], tensor_cores=tc)
            e1.record(s)
            torch.cuda.synchronize()
            out[name + "_ms"] = round(e0.elapsed_time(e1) / reps, 3)
        d = (tc_logits[:n] - self.logits[:n]).abs()
        out.update({"candidates": n, "max_abs_logit_diff": round(float(d.max()), 5),
                    "frac_within_1e-3": round(float((d <= 1e-3).float().mean()), 4), "tc_status": self.clf.status()})
        return out


def run_rfi(P, dev, reps=10):
    """Coincidence RFI mask over 13 beams of the single-beam gulp shape (1024
    channels x 2^19 + maxdelay samples each, 1.8 GB in), 3 sigma in >= 4 beams,
    masked samples substituted in place; a coincident broadband burst is
    injected into 6 beams."""
    import torch

    f = synth.band_freqs(NCHAN)
    nsamp = NOUT + 20464
    beams = []
    for b in range(13):
        d = synth.device_noise_packed(NCHAN, nsamp, seed=synth.BASE_SEED + 6000 + b, device=dev)
        if b < 6:
            rec = synth.BeamRecipe(bursts=[synth.Burst(t=123456, dur=500)])
            synth.device_apply_recipe(d, nsamp, rec)
        beams.append(d)
    r = P.RfiMask(13, NCHAN, nsamp)
    r.run(beams, nsamp, apply=True)
    nm = r.nmasked()   # the burst, now replaced in place: the timed runs find nothing to substitute
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        r.run(beams, nsamp, apply=True)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    r.close()
    del f
    in_bytes = 13 * NCHAN * beams[0].shape[1]
    return {"beams": 13, "nsamp": nsamp, "ms": round(ms, 3), "gsamps": round(13 * NCHAN * nsamp / ms / 1e6, 1),
            "input_gbs": round(in_bytes / ms / 1e6, 1), "masked_samples_first_run": nm,
            "rule": "3 sigma in >= 4 beams"}


def run_multibeam(P, dev, clf_unused=None, replays=10):
    """13 beams of uneven gulps and DM ranges in one persistent launch
    replayed from a CUDA graph."""
    import torch

    rng = np.random.default_rng(synth.BASE_SEED + 3000)
    f = synth.band_freqs(NCHAN)
    plans, items = {}, []
    for b in range(13):
        nout = int(rng.integers(1 << 16, (1 << 19) + 1))
        dm_max = float(rng.choice([250.0, 500.0, 1000.0]))
        if dm_max not in plans:
            plans[dm_max] = P.Plan(f, TSAMP, synth.dm_list_piecewise(dm_max))
        plan = plans[dm_max]
        nsamp = nout + plan.maxdelay
        d_in = beam_gulp(NCHAN, nsamp, nout, dm_max, synth.BASE_SEED + 3000 + b,
                         lambda dm: P.compute_delays(f, TSAMP, [dm])[0], dev)
        items.append((plan, d_in, nsamp, plan.alloc_output(nsamp, dev)))
    batch = P.Batch(items, use_graph=True)
    info = batch.info()
    batch.launch()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(replays):
        batch.launch()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / replays
    samples = sum(p.nchan * p.ndm * p.nout(ns) for p, _, ns, _ in items)
    data_s = [p.nout(ns) * TSAMP for p, _, ns, _ in items]
    rep = {"beams": 13, "ms_per_launch": round(ms, 3), "gsamps": round(samples / (ms / 1e3) / 1e9, 1),
           "tiles": info["ntiles"], "grid": info["grid"], "graph": True,
           "realtime_factor_min": round(min(data_s) / (ms / 1e3), 1),
           "all_beams_realtime": bool(min(data_s) > ms / 1e3)}
    batch.close()
    del items
    return rep


def run_serving(P, dev, minutes=10.0, accel=30.0, gulp_log2=17, clf_path=None, seed=synth.BASE_SEED + 5000):
    """13 beams stream 2^17-sample gulps (8.39 s of data each) with +-10%
    arrival jitter over a simulated observation, replayed `accel` times faster
    than real time through the streaming server; then the same gulps as fast
    as the server admits them (sustained real-time factor)."""
    import torch

    G = 1 << gulp_log2
    f = synth.band_freqs(NCHAN)
    dm_of_beam = [(250.0, 500.0, 1000.0)[b % 3] for b in range(13)]
    plans = {dm: P.Plan(f, TSAMP, synth.dm_list_piecewise(dm)) for dm in set(dm_of_beam)}
    pool = []  # per beam: 2 pinned host gulps (cycled)
    for b in range(13):
        g = []
        for k in range(2):
            d = beam_gulp(NCHAN, G, G - 1, dm_of_beam[b], seed + 10 * b + k,
                          lambda dm: P.compute_delays(f, TSAMP, [dm])[0], dev)
            h = torch.empty((NCHAN, G // 4), dtype=torch.uint8, pin_memory=True)
            h.copy_(d[:, :G // 4])
            g.append(h)
        pool.append(g)
    gulp_s = G * TSAMP
    ngulps = int(np.ceil(minutes * 60.0 / gulp_s))
    rng = np.random.default_rng(seed)
    arrivals = []
    for b in range(13):
        t = 0.0
        for k in range(ngulps):
            t += gulp_s * rng.uniform(0.9, 1.1)
            arrivals.append((t, b, k))
    arrivals.sort()

    def replay(speed):
        srv = P.Server([plans[dm] for dm in dm_of_beam], G, max_slots=16, half_window=4096, widths=WIDTHS,
                       thresh=6.0, max_cands=16384, classifier_path=clf_path, nn_batch=4096)
        # warm-up: one gulp per beam creates the slots
        for b in range(13):
            while srv.submit(b, pool[b][0]) is None:
                srv.poll(wait_s=0.05)
        srv.drain()
        srv.poll(max_results=64)
        srv.close()
        srv = P.Server([plans[dm] for dm in dm_of_beam], G, max_slots=16, half_window=4096, widths=WIDTHS,
                       thresh=6.0, max_cands=16384, classifier_path=clf_path, nn_batch=4096)
        t_start = time.monotonic()  # the server stamps completions with the same monotonic clock
        lat, ncand, done = [], 0, 0
        i = 0
        pending = []
        arrive_at = {}
        while done < len(arrivals):
            now = time.monotonic() - t_start
            while i < len(arrivals) and (speed is None or arrivals[i][0] / speed <= now):
                pending.append(arrivals[i])
                i += 1
            while pending:
                t, b, k = pending[0]
                seq = srv.submit(b, pool[b][k % 2])
                if seq is None:
                    break
                arrive_at[(b, seq)] = t_start + (t / speed if speed else 0.0)
                pending.pop(0)
            for r, c in srv.poll(wait_s=0.002, max_results=64):
                lat.append(r["t_done"] - arrive_at.pop((r["beam"], r["seq"])))
                ncand += len(c)
                done += 1
        wall = time.monotonic() - t_start
        srv.close()
        return lat, wall, ncand

    lat, wall_rt, nc = replay(accel)
    _, wall_sat, _ = replay(None)
    data_s = 13 * ngulps * gulp_s
    lat_ms = np.array(lat) * 1e3
    return {"beams": 13, "gulp_samples": G, "gulp_s": round(gulp_s, 3), "gulps_per_beam": ngulps,
            "simulated_minutes": minutes, "arrival_speedup": accel,
            "latency_ms_p50": round(float(np.percentile(lat_ms, 50)), 2),
            "latency_ms_p99": round(float(np.percentile(lat_ms, 99)), 2),
            "latency_ms_max": round(float(lat_ms.max()), 2),
            "candidates": int(nc), "sustained_realtime_factor": round(data_s / wall_sat, 1),
            "all_beams_realtime": bool(data_s / wall_sat > 1.0)}


def run_gpu(args):
    import torch

    import paper_1112_0065_gb300 as P
    from paper_1112_0065_gb300 import probes

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    f = synth.band_freqs(NCHAN)
    dms = synth.dm_list_piecewise(1000.0)
    plan = P.Plan(f, TSAMP, dms)
    nsamp = NOUT + plan.maxdelay
    ld_in = P.row_bytes(nsamp)
    offsets = lambda dm: P.compute_delays(f, TSAMP, [dm])[0]  # noqa: E731
    # every rank processes its own beam: two rotating gulps (2 x 139.5 MB) with
    # pulses and RFI, 3.15 GB of dedispersed output and ~11 GB of search
    # buffers per step -- far more than the 129 MB L2, so no explicit flush
    gulps = [beam_gulp(NCHAN, nsamp, NOUT, 1000.0, synth.BASE_SEED + 100 * rank + k, offsets, dev)
             for k in range(2)]
    tune_ms = plan.autotune(nsamp)
    shape = plan.kernel_shape()
    clf = P.Classifier(max_batch=CLF_BATCH, seed=1)
    pipe = GulpPipeline(P, plan, NOUT, clf, dev)
    stream = torch.cuda.current_stream(dev)

    for k in range(max(args.warmup, 3)):
        pipe.step(gulps[k % 2])
    torch.cuda.synchronize(dev)

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    launches = 0
    ncands = []
    nhots = []
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for k in range(args.steps):
            launches += pipe.step(gulps[k % 2], evs[k])
            ncands.append(pipe.last_n)
            nhots.append(pipe.last_nhot)
        t_end.record(stream)
        torch.cuda.synchronize(dev)
    rebuilds = pipe.search.stats()["median_rebuilds"]   # of the last step's search
    if ws > 1:
        torch.distributed.barrier()
    total_ms = t_start.elapsed_time(t_end)
    stage_ms = np.array([[e[i].elapsed_time(e[i + 1]) for i in range(4)] for e in evs])
    if ws > 1:
        import torch.distributed as dist

        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())

    samples_per_step = NCHAN * len(dms) * NOUT
    value = ws * samples_per_step * args.steps / (total_ms / 1e3) / 1e9
    kern_ms = stage_ms[:, 0]

    # dedispersion alone, back to back (the kernel the roofline is about)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        plan.execute(gulps[k % 2], nsamp, pipe.out)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    dd_only_ms = e0.elapsed_time(e1) / args.steps
    clf_variants = pipe.classifier_variants() if not args.skip_extras else None
    base_variants = pipe.baseline_variants() if not args.skip_extras else None

    # end to end through the public streaming API: pinned host gulps in,
    # candidates out, the device carrying the overlap between gulps
    e2e = None
    if rank == 0:
        import tempfile

        tmpd = tempfile.mkdtemp()
        ckpt = os.path.join(tmpd, "clf.ckpt")
        clf.save(ckpt)
        h = [torch.empty((NCHAN, NOUT // 4), dtype=torch.uint8, pin_memory=True) for _ in range(2)]
        for k in range(2):
            h[k].copy_(gulps[k][:, :NOUT // 4])
        del pipe
        torch.cuda.empty_cache()
        srv = P.Server([plan], NOUT, max_slots=3, half_window=4096, widths=WIDTHS, thresh=6.0, max_cands=1 << 17,
                       classifier_path=ckpt, nn_batch=CLF_BATCH)
        n_e2e = max(3, min(args.steps, 20))
        cand_bytes = 0
        for k in range(3):  # warm-up: slot creation
            while srv.submit(0, h[k % 2]) is None:
                srv.poll(wait_s=0.05)
        srv.drain()
        srv.poll(max_results=8)
        t0 = time.perf_counter()
        done = 0
        k = 0
        while done < n_e2e:
            if k < n_e2e and srv.submit(0, h[k % 2]) is not None:
                k += 1
            for r, c in srv.poll(wait_s=0.001):
                done += 1
                cand_bytes += len(c) * 32
        wall = (time.perf_counter() - t0) / n_e2e
        srv.close()
        e2e = {"value": round(samples_per_step / wall / 1e9, 3), "unit": "Gsamp/s",
               "h2d_bytes_per_step": NCHAN * NOUT // 4, "d2h_bytes_per_step": int(cand_bytes / n_e2e),
               "api": "dd_server_submit/dd_server_poll (pinned host gulps of 2^19 new samples; device-carried "
                      "overlap; dedispersion, search, snippets, classifier; candidates to host)"}
    line = None
    if rank == 0:
        peaks, peak_src = measured_peaks()
        clocks = clk.summary()
        avg_kern_s = float(np.mean(kern_ms)) / 1e3
        achieved = samples_per_step / avg_kern_s / 1e12
        peak = alu_peak_tadds(float(peaks.get("sm_max_mhz", 2070.0)))
        traffic = profiled_traffic((shape[1], shape[2], shape[3]))
        bytes_algo = NCHAN * ld_in + len(dms) * NOUT * 4
        probe = {k: round(v, 2) for k, v in probes.int_rates().items()}
        fp = probes.fp_rates()
        clf_ms = float(np.mean(stage_ms[:, 3]))
        clf_achieved = float(np.mean(ncands)) * CLF_MAC_PER_SNIPPET / (clf_ms / 1e3) / 1e12
        multibeam = run_multibeam(P, dev) if not args.skip_extras else None
        rfi = run_rfi(P, dev) if not args.skip_extras else None
        serving = run_serving(P, dev, minutes=args.serve_minutes, accel=args.serve_accel, clf_path=ckpt) \
            if not args.skip_extras else None
        clf_eval = None
        if not (args.skip_extras or args.no_classifier_eval):
            from paper_1112_0065_gb300 import training

            clf_eval = training.evaluate(log=lambda *a: None)
            clf_eval.pop("eval_per_gulp", None)
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "Gsamp/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "step": "dedispersion + running-median baseline + boxcar matched "
                       "filter (1..1024) + S/N>=6 grouping + snippets + classifier scores, per gulp",
                       "nchan": NCHAN, "ndm": len(dms), "nsamp_out": NOUT, "nsamp_in": nsamp,
                       "maxdelay": plan.maxdelay, "beams_per_gpu": 1,
                       "injection": "20 dispersed pulses, 5% stuck channels, 3 zero-DM bursts per gulp",
                       "l2": "inputs larger than L2 (2 rotating 139.5 MB gulps, 3.15 GB output, ~11 GB search "
                             "buffers per step), no flush",
                       "kernel_shape": {"kernel": shape[0], "dms_per_block": shape[1],
                                        "words_per_thread": shape[2], "chan_chunk": shape[3]},
                       "autotune_best_ms": round(tune_ms, 4)},
            "stages_ms": {"dedisperse": round(float(np.mean(stage_ms[:, 0])), 3),
                          "search": round(float(np.mean(stage_ms[:, 1])), 3),
                          "count+snippets": round(float(np.mean(stage_ms[:, 2])), 3),
                          "classifier": round(float(np.mean(stage_ms[:, 3])), 3),
                          "candidates_per_gulp": int(np.mean(ncands)),
                          "hot_cells_per_gulp": int(np.mean(nhots)),
                          "median_rebuilds_per_gulp": rebuilds},
            "classifier_variants": clf_variants,
            "baseline_variants": base_variants,
            "dedisp_only": {"ms": round(dd_only_ms, 4), "gsamps": round(samples_per_step / dd_only_ms / 1e6, 1),
                            "realtime_factor": round(NOUT * TSAMP / (dd_only_ms / 1e3), 1)},
            "roofline": {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 3), "unit": "Tadd/s",
                         "frac": round(achieved / peak, 4), "traffic": traffic,
                         "peak_source": ("of measured: 152 SMs x 128 INT32 add lanes x sm_max_mhz "
                                         "(MEASURED_PEAKS.json)") if peak_src == "measured" else "of fallback",
                         "kernel": "dd_tiled_kernel", "kernel_ms": round(avg_kern_s * 1e3, 4),
                         "int_issue_probe_tops": probe,
                         "hbm_frac": round(bytes_algo / avg_kern_s / 1e9 / float(peaks.get("hbm_gbs", 6800.0)), 4),
                         "realtime_factor": round(NOUT * TSAMP / avg_kern_s, 2)},
            "classifier_roofline": {
                "bound": "fma", "achieved": round(clf_achieved, 3), "peak": round(fp["ffma2"], 3), "unit": "T FMA/s",
                "frac": round(clf_achieved / fp["ffma2"], 4),
                "peak_source": "of measured: dd_probe_fp_rates, packed fma.rn.f32x2 on this GPU",
                "work": "%d multiply-adds per snippet (4 convolutions + 2 fc layers) x candidates per gulp, "
                        "over the classifier stage's time" % CLF_MAC_PER_SNIPPET,
                "kernels": "conv_fwd_kernel, fc1_persist_kernel, fc2_fwd_kernel (fixed-order float FMAs: the "
                           "summation order that makes logits bit-exact runs on the FMA pipe, not the tensor cores)"},
            "multibeam": multibeam,
            "rfi_mask": rfi,
            "serving": serving,
            "classifier_eval": clf_eval,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
        }
    if ws > 1:
        torch.distributed.barrier()
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    plan.close()
    return 0


def run_ncu_search_case(args):
    """Small case for an ncu capture of the search kernels: the single-beam
    band and DM list with 2^17 output samples and the injection recipe, one
    warm-up search and one more.  With --ncu-half-window 1024 the median
    kernel has as many lane slots (and warps) as on a full 2^19-sample gulp
    with the default half window."""
    import torch

    import paper_1112_0065_gb300 as P

    f = synth.band_freqs(NCHAN)
    dms = synth.dm_list_piecewise(1000.0)
    plan = P.Plan(f, TSAMP, dms)
    nout = 1 << 17
    nsamp = nout + plan.maxdelay
    d_in = beam_gulp(NCHAN, nsamp, nout, 1000.0, synth.BASE_SEED, lambda dm: P.compute_delays(f, TSAMP, [dm])[0],
                     "cuda")
    x = plan.execute(d_in, nsamp)
    s = P.Search(len(dms), nout, nchan=NCHAN, half_window=args.ncu_half_window, widths=WIDTHS, thresh=6.0,
                 max_cands=1 << 16, full_map=False, baseline=args.ncu_baseline)
    for _ in range(2):
        s.run(x, len(dms), nout)
        n = min(s.result()["ngroups"], 1 << 16)
        s.snippets(n)
    torch.cuda.synchronize()
    print("ncu search case done", s.result(), s.stats())
    return 0


def run_ncu_nn_case(args):
    """Small case for an ncu capture of the classifier kernels: forward passes
    over 8192 random bfloat16 snippets with seeded weights, one warm-up and
    two more."""
    import torch

    import paper_1112_0065_gb300 as P

    clf = P.Classifier(max_batch=NCU_NN_BATCH, seed=synth.BASE_SEED)
    g = torch.Generator(device="cuda").manual_seed(synth.BASE_SEED)
    x = torch.randn((NCU_NN_BATCH, 64, 64), generator=g, device="cuda").to(torch.bfloat16)
    for _ in range(3):
        clf.forward(x)
    torch.cuda.synchronize()
    print("ncu nn case done")
    return 0


def run_ncu_case(args):
    """Small case for an ncu capture of the tiled kernel: the single-beam band
    and DM list with 2^18 output samples (72 MB in, 1.5 GB out), one warm-up
    launch and two more, default tile shape."""
    import torch

    import paper_1112_0065_gb300 as P

    f = synth.band_freqs(NCHAN)
    dms = synth.dm_list_piecewise(1000.0)
    plan = P.Plan(f, TSAMP, dms, kernel=P.KERNEL_TILED, dms_per_block=args.ncu_dpb, words_per_thread=args.ncu_w,
                  chan_chunk=args.ncu_g)
    nsamp = (1 << 18) + plan.maxdelay
    d_in = synth.device_noise_packed(NCHAN, nsamp, seed=synth.BASE_SEED)
    out = plan.alloc_output(nsamp)
    for _ in range(3):
        plan.execute(d_in, nsamp, out)
    torch.cuda.synchronize()
    print("ncu case done", plan.kernel_shape())
    return 0


def shape_table(args) -> int:
    """Time every tiled shape (DMs per CTA x words per lane x channels per
    stage) on the single-beam workload (1024 ch x 1500 DM x 2^19 samples)
    and print the table, fastest first, with the autotuner's own choice."""
    import torch

    import paper_1112_0065_gb300 as P

    f = synth.band_freqs(NCHAN)
    dms = synth.dm_list_piecewise(1000.0)
    auto = P.Plan(f, TSAMP, dms)
    nsamp = NOUT + auto.maxdelay
    d_in = synth.device_noise_packed(NCHAN, nsamp, seed=synth.BASE_SEED)
    out = auto.alloc_output(nsamp)
    auto.autotune(nsamp)
    rows = []
    for g in (32, 64, 128):
        for dt, w in ((1, 2), (2, 1), (2, 2), (4, 1), (1, 4), (1, 3), (2, 3), (1, 5)):
            plan = P.Plan(f, TSAMP, dms, kernel=P.KERNEL_TILED, dms_per_block=8 * dt, words_per_thread=w,
                          chan_chunk=g)
            for _ in range(2):
                plan.execute(d_in, nsamp, out)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(5):
                plan.execute(d_in, nsamp, out)
            e1.record()
            torch.cuda.synchronize()
            rows.append((e0.elapsed_time(e1) / 5, 8 * dt, w, g))
            plan.close()
    _, dpb, w, g = auto.kernel_shape()
    print("| DMs per CTA | words per lane (x16 samples) | channels per stage | ms | Gsamp/s |\n|---|---|---|---|---|")
    for ms, d, ww, gg in sorted(rows):
        mark = " (tuned)" if (d, ww, gg) == (dpb, w, g) else ""
        print(f"| {d} | {ww} | {gg} | {ms:.3f}{mark} | {NCHAN * len(dms) * NOUT / ms / 1e6:.0f} |")
    return 0


def launch_table(path: str) -> int:
    """Per-step table of an ncu launch list (``--metrics gpu__time_duration.sum
    --csv`` of this bench): every kernel's launches and device time per step,
    steps counted by the median-baseline launches (one per gulp); of the
    dedispersion kernels only the shape launched most often (the autotuner's
    choice, once per gulp) is kept; PyTorch and library kernels of the input
    generator are left out."""
    import collections
    import csv
    import re

    hdr, agg = None, collections.OrderedDict()
    with open(path) as fh:
        for r in csv.reader(fh):
            if r and r[0] == "ID":
                hdr = r
                continue
            if not hdr or len(r) != len(hdr):
                continue
            d = dict(zip(hdr, r))
            if d.get("Metric Name") != "gpu__time_duration.sum":
                continue
            full = re.sub(r"\(.*", "", d["Kernel Name"]).replace("void ", "")
            if full.startswith(("at::", "at_cuda_detail::", "cub::", "select::", "reduce::", "scan::")):
                continue  # PyTorch's and CUB's own kernels (the synthetic-input generator)
            name = re.sub(r"^((\w+|<unnamed>)::)+", "", full)  # drop the namespaces
            v = float(d["Metric Value"].replace(",", "")) * {"ns": 1e-6, "us": 1e-3, "ms": 1.0}[d["Metric Unit"]]
            a = agg.setdefault(name, [0, 0.0])
            a[0] += 1
            a[1] += v
    steps = sum(n for k, (n, _) in agg.items() if k.startswith("dd_median_kernel"))
    tiled = [k for k in agg if k.startswith("dd_tiled_kernel")]
    chosen = max(tiled, key=lambda k: agg[k][0]) if tiled else None
    rows = {}
    for k, (n, t) in agg.items():
        if k.startswith("dd_tiled_kernel"):
            if k == chosen:
                rows[k] = (t / n, 1.0)
        elif not (k.startswith("probe_kernel") or "elementwise" in k or "distribution" in k):
            rows[k] = (t / steps, n / steps)
    tot = sum(v[0] for v in rows.values())
    print("| kernel | launches per step | ms per step | share |\n|---|---|---|---|")
    for k, (ms, nl) in sorted(rows.items(), key=lambda x: -x[1][0]):
        print(f"| {k} | {nl:g} | {ms:.3f} | {100 * ms / tot:.1f} % |")
    print(f"| total | | {tot:.3f} | 100 % |")
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ncu-case", action="store_true", help="small fixed case for profiling, no timing")
    ap.add_argument("--ncu-search-case", action="store_true", help="small fixed search case for profiling")
    ap.add_argument("--ncu-nn-case", action="store_true", help="small fixed classifier case for profiling")
    ap.add_argument("--skip-extras", action="store_true",
                    help="skip the multibeam, RFI, serving, classifier-evaluation and variant sections")
    ap.add_argument("--no-classifier-eval", action="store_true",
                    help="skip the held-out classifier evaluation (about a minute of training)")
    ap.add_argument("--serve-minutes", type=float, default=10.0)
    ap.add_argument("--serve-accel", type=float, default=10.0)
    ap.add_argument("--ncu-dpb", type=int, default=16)
    ap.add_argument("--ncu-w", type=int, default=2)
    ap.add_argument("--ncu-g", type=int, default=64, help="channels per stage of the ncu case")
    ap.add_argument("--shape-table", action="store_true",
                    help="time every tiled shape on the single-beam workload and print the table")
    ap.add_argument("--ncu-baseline", default="median", choices=["median", "mean"],
                    help="baseline of the search case")
    ap.add_argument("--launch-table", metavar="CSV", help="print the per-step table of an ncu launch list and exit")
    ap.add_argument("--ncu-half-window", type=int, default=4096,
                    help="baseline half window of the search case (1024 gives the full gulp's median grid)")
    args = ap.parse_args()
    if args.launch_table:
        return launch_table(args.launch_table)
    if args.shape_table:
        return shape_table(args)
    if args.ncu_case:
        return run_ncu_case(args)
    if args.ncu_search_case:
        return run_ncu_search_case(args)
    if args.ncu_nn_case:
        return run_ncu_nn_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
