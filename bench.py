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
KERNEL_SRC = os.path.join(ROOT, "paper_1112_0065_gb300", "csrc", "dedisp_kernels.cu")
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "dd_tiled_kernel_htru_1024x1500.md")


def kernel_source_hash() -> str:
    with open(KERNEL_SRC, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def alu_peak_tadds(sm_mhz: float, sms: int = 152) -> float:
    """INT32 add peak: 152 SMs x 128 INT32 lanes per SM per clock x SM clock."""
    return sms * 128 * sm_mhz * 1e6 / 1e12


def profiled_traffic():
    """DRAM bytes per launch recorded by the committed ncu summary, if it was
    taken on the current kernel source."""
    if not os.path.exists(PROFILE_SUMMARY):
        return None
    src_hash = kernel_source_hash()
    h = t = None
    with open(PROFILE_SUMMARY) as f:
        for line in f:
            if line.startswith("kernel_source_sha256_16:"):
                h = line.split(":", 1)[1].strip()
            if line.startswith("dram_bytes_per_launch:"):
                t = float(line.split(":", 1)[1].strip())
    return t if (h == src_hash and t is not None) else None


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


def cpu_oracle_run(ndm_sample: int, seed: int = 1):
    """Time the oracle on a bounded sample of the workload: ndm_sample of the
    1500 trial DMs (evenly spaced) over the full 2^19-sample gulp."""
    import oracle

    f = synth.band_freqs(NCHAN)
    dms_all = synth.dm_list_piecewise(1000.0)
    delays_all = oracle.delay_table(f, TSAMP, dms_all)
    maxdelay = int(delays_all.max())
    nsamp = NOUT + maxdelay
    if seed not in _HOST_GULP:
        _HOST_GULP[seed] = synth.noise_packed(np.random.default_rng(seed), NCHAN, nsamp)
    packed = _HOST_GULP[seed]
    idx = np.linspace(0, 1499, ndm_sample).round().astype(int)
    idx[-1] = 1499  # keep the largest delay so the output length is the workload's
    delays = np.ascontiguousarray(delays_all[idx])
    t0 = time.perf_counter()
    out = oracle.dedisperse(delays, packed, nsamp)
    dt = time.perf_counter() - t0
    assert out.shape == (ndm_sample, NOUT)
    return NCHAN * ndm_sample * NOUT / dt / 1e9, dt, oracle.num_threads()


def cpu_baseline(target_s: float = 10.0):
    gs, dt, thr = cpu_oracle_run(16)
    n = int(max(16, min(1500, round(16 * target_s / max(dt, 1e-3)))))
    n = max(16, (n // 16) * 16)
    if n > 16:
        gs, dt, thr = cpu_oracle_run(n)
    return {"value": round(gs, 4), "unit": "Gsamp/s", "cores": thr, "kind": "oracle",
            "sample": f"{n} of 1500 DM trials (evenly spaced, incl. DM 999) x 1024 ch x 2^19 samples; "
                      f"{dt:.1f} s of CPU work"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    cb = cpu_baseline(target_s=max(2.0, min(20.0, 60.0 / max(args.steps + args.warmup, 1))))
    vals = []
    n = int(cb["sample"].split()[0])
    for _ in range(args.warmup):
        cpu_oracle_run(n)
    t_all = 0.0
    for _ in range(args.steps):
        gs, dt, _ = cpu_oracle_run(n)
        vals.append(gs)
        t_all += dt
    value = float(np.mean(vals)) if vals else cb["value"]
    cb["value"] = round(value, 4)
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "Gsamp/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * t_all / max(args.steps, 1), 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": WORKLOAD + " (oracle on a DM-trial sample per step)", "nchan": NCHAN,
                       "ndm": 1500, "nsamp_out": NOUT},
            "cpu_baseline": cb,
            "e2e": {"value": round(value, 4), "unit": "Gsamp/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_gpu(args):
    import torch

    import paper_1112_0065_gb300 as P

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
    # two rotating gulps (2 x 139.5 MB) and the 3.15 GB output: the working set
    # per step is far larger than the 129 MB L2, so no explicit flush is needed
    gulps = [synth.device_noise_packed(NCHAN, nsamp, seed=synth.BASE_SEED + 100 * rank + k, device=dev)
             for k in range(2)]
    out = plan.alloc_output(nsamp, dev)
    tune_ms = plan.autotune(nsamp)
    shape = plan.kernel_shape()
    stream = torch.cuda.current_stream(dev)

    for k in range(max(args.warmup, 3)):
        plan.execute(gulps[k % 2], nsamp, out)
    torch.cuda.synchronize(dev)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for k in range(args.steps):
            ev[k][0].record(stream)
            plan.execute(gulps[k % 2], nsamp, out)
            ev[k][1].record(stream)
        t_end.record(stream)
        torch.cuda.synchronize(dev)
    if ws > 1:
        torch.distributed.barrier()
    total_ms = t_start.elapsed_time(t_end)
    kern_ms = [a.elapsed_time(b) for a, b in ev]
    if ws > 1:
        import torch.distributed as dist

        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())

    samples_per_step = NCHAN * len(dms) * NOUT
    value = ws * samples_per_step * args.steps / (total_ms / 1e3) / 1e9

    # end to end through the C ABI with host buffers (pinned): H2D of the gulp,
    # dedispersion, D2H of the whole uint32 result, every step
    h_in = torch.empty((NCHAN, ld_in), dtype=torch.uint8, pin_memory=True)
    h_in.copy_(gulps[0].cpu())
    h_out = torch.empty((len(dms), P.out_stride(NOUT)), dtype=torch.int32, pin_memory=True)
    e2e_steps = max(2, min(args.steps, 5))
    plan.execute_host(h_in, nsamp, h_out)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        plan.execute_host(h_in, nsamp, h_out)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_val = samples_per_step / e2e_s / 1e9

    line = None
    if rank == 0:
        peaks, peak_src = measured_peaks()
        clocks = clk.summary()
        avg_kern_s = float(np.mean(kern_ms)) / 1e3
        achieved = samples_per_step / avg_kern_s / 1e12
        peak = alu_peak_tadds(float(peaks.get("sm_max_mhz", 2070.0)))
        traffic = profiled_traffic()
        bytes_algo = NCHAN * ld_in + len(dms) * NOUT * 4
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "Gsamp/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nchan": NCHAN, "ndm": len(dms), "nsamp_out": NOUT,
                       "nsamp_in": nsamp, "maxdelay": plan.maxdelay, "beams_per_gpu": 1,
                       "l2": "inputs larger than L2 (2 rotating 139.5 MB gulps + 3.15 GB output), no flush",
                       "kernel_shape": {"kernel": shape[0], "dms_per_block": shape[1],
                                        "words_per_thread": shape[2], "chan_chunk": shape[3]},
                       "autotune_best_ms": round(tune_ms, 4)},
            "roofline": {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 3), "unit": "Tadd/s",
                         "frac": round(achieved / peak, 4), "traffic": traffic,
                         "peak_source": "152 SMs x 128 INT32 lanes x sm_max_mhz from MEASURED_PEAKS.json"
                                        if peak_src == "measured" else "fallback clocks",
                         "kernel": "dd_tiled_kernel", "kernel_ms": round(avg_kern_s * 1e3, 4),
                         "hbm_frac": round(bytes_algo / avg_kern_s / 1e9 / float(peaks.get("hbm_gbs", 6800.0)), 4),
                         "realtime_factor": round(NOUT * TSAMP / avg_kern_s, 2)},
            "e2e": {"value": round(e2e_val, 3), "unit": "Gsamp/s", "h2d_bytes_per_step": NCHAN * ld_in,
                    "d2h_bytes_per_step": len(dms) * P.out_stride(NOUT) * 4},
            "gpu_launches": args.steps,
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


def run_ncu_case(args):
    """Small case for an ncu capture of the tiled kernel: the single-beam band
    and DM list with 2^18 output samples (72 MB in, 1.5 GB out), one warm-up
    launch and two more, default tile shape."""
    import torch

    import paper_1112_0065_gb300 as P

    f = synth.band_freqs(NCHAN)
    dms = synth.dm_list_piecewise(1000.0)
    plan = P.Plan(f, TSAMP, dms, kernel=P.KERNEL_TILED, dms_per_block=args.ncu_dpb, words_per_thread=args.ncu_w)
    nsamp = (1 << 18) + plan.maxdelay
    d_in = synth.device_noise_packed(NCHAN, nsamp, seed=synth.BASE_SEED)
    out = plan.alloc_output(nsamp)
    for _ in range(3):
        plan.execute(d_in, nsamp, out)
    torch.cuda.synchronize()
    print("ncu case done", plan.kernel_shape())
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ncu-case", action="store_true", help="small fixed case for profiling, no timing")
    ap.add_argument("--ncu-dpb", type=int, default=16)
    ap.add_argument("--ncu-w", type=int, default=2)
    args = ap.parse_args()
    if args.ncu_case:
        return run_ncu_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
