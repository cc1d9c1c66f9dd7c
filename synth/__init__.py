"""Seeded synthetic filterbank generator shared by the tests, the benchmark and
the serving demo.

It produces 2-bit filterbank gulps shaped like the Parkes HTRU backend the
paper describes (Section 1: 1024 channels over 400 MHz centred at 1381.8 MHz,
64 us sampling, 2 bits per sample, 13 beams).  It holds none of the
dedispersion arithmetic: where a dispersed pulse is injected, the caller
passes the per-channel arrival offsets in.

Conventions
-----------
* Channel frequencies are channel centres, highest first.
* A sample is N(0, 1) quantised at (-0.98, 0, 0.98): the level is the number
  of thresholds at or below it, 0..3.  The level is drawn from a uniform 32-bit
  integer with cut points at the normal CDF of the thresholds, which has the
  same distribution.
* Packing is channel-major, 4 samples per byte along time, the earliest
  sample in the least-significant bits; rows are padded to a multiple of 16
  bytes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

TSAMP_HTRU = 64e-6
F_TOP_HTRU = 1581.8
BW_HTRU = 400.0
QUANT_THRESHOLDS = (-0.98, 0.0, 0.98)
BASE_SEED = 11120065


def _phi(x: float) -> float:
    return 0.5 * math.erfc(-x / math.sqrt(2.0))


# Uniform-integer cut points equivalent to quantising N(0,1) at the thresholds.
_CUTS32 = np.array([min(int(round(_phi(th) * 2.0**32)), 2**32 - 1) for th in QUANT_THRESHOLDS],
                   dtype=np.uint64)


def level_probabilities():
    p = [_phi(QUANT_THRESHOLDS[0]), _phi(QUANT_THRESHOLDS[1]) - _phi(QUANT_THRESHOLDS[0]),
         _phi(QUANT_THRESHOLDS[2]) - _phi(QUANT_THRESHOLDS[1]), 1.0 - _phi(QUANT_THRESHOLDS[2])]
    return np.array(p)


def band_freqs(nchan: int, f_top: float = F_TOP_HTRU, bw: float = BW_HTRU) -> np.ndarray:
    """Channel-centre frequencies (MHz), highest first."""
    df = bw / nchan
    return f_top - (np.arange(nchan, dtype=np.float64) + 0.5) * df


def dm_list_linear(ndm: int, dm_end: float) -> np.ndarray:
    """ndm trials i*dm_end/ndm (half-open grid, so dm_end/2 is trial ndm/2)."""
    return np.arange(ndm, dtype=np.float64) * (dm_end / ndm)


def dm_list_piecewise(dm_end: float = 1000.0) -> np.ndarray:
    """Step 0.25 over [0,100), 0.5 over [100,300), 1.0 over [300,dm_end)."""
    parts = []
    for lo, hi, step in ((0.0, 100.0, 0.25), (100.0, 300.0, 0.5), (300.0, 1e30, 1.0)):
        hi = min(hi, dm_end)
        if hi <= lo:
            break
        n = int(round((hi - lo) / step))
        parts.append(lo + step * np.arange(n, dtype=np.float64))
    return np.concatenate(parts)


def padded_row_bytes(nsamp: int) -> int:
    nbytes = (nsamp + 3) // 4
    return (nbytes + 15) // 16 * 16


def noise_levels(rng: np.random.Generator, nchan: int, nsamp: int) -> np.ndarray:
    u = rng.integers(0, 2**32, size=(nchan, nsamp), dtype=np.uint64)
    lv = (u >= _CUTS32[0]).astype(np.uint8)
    lv += (u >= _CUTS32[1])
    lv += (u >= _CUTS32[2])
    return lv


def noise_packed(rng: np.random.Generator, nchan: int, nsamp: int, ld_bytes: int | None = None) -> np.ndarray:
    """Packed quantised noise generated a few channels at a time (bounded host
    memory); same draws as pack2(noise_levels(rng, nchan, nsamp))."""
    if ld_bytes is None:
        ld_bytes = padded_row_bytes(nsamp)
    out = np.empty((nchan, ld_bytes), dtype=np.uint8)
    rows = max(1, (1 << 24) // max(nsamp, 1))
    for c0 in range(0, nchan, rows):
        c1 = min(nchan, c0 + rows)
        out[c0:c1] = pack2(noise_levels(rng, c1 - c0, nsamp), ld_bytes)
    return out


def pack2(levels: np.ndarray, ld_bytes: int | None = None) -> np.ndarray:
    """uint8 levels [nchan, nsamp] (0..3) -> packed uint8 [nchan, ld_bytes]."""
    levels = np.asarray(levels, dtype=np.uint8)
    nchan, nsamp = levels.shape
    if ld_bytes is None:
        ld_bytes = padded_row_bytes(nsamp)
    pad = ld_bytes * 4 - nsamp
    if pad < 0:
        raise ValueError("ld_bytes too small")
    lv = np.zeros((nchan, ld_bytes * 4), dtype=np.uint8)
    lv[:, :nsamp] = levels & 3
    lv = lv.reshape(nchan, ld_bytes, 4)
    return (lv[:, :, 0] | (lv[:, :, 1] << 2) | (lv[:, :, 2] << 4) | (lv[:, :, 3] << 6)).astype(np.uint8)


def unpack2(packed: np.ndarray, nsamp: int) -> np.ndarray:
    packed = np.asarray(packed, dtype=np.uint8)
    out = np.stack([(packed >> (2 * k)) & 3 for k in range(4)], axis=-1)
    return out.reshape(packed.shape[0], -1)[:, :nsamp]


@dataclass
class Pulse:
    t0: int            # arrival sample in the highest-frequency channel
    offsets: np.ndarray  # per-channel arrival offset (samples), supplied by the caller
    amp: int           # levels added (clipped at 3)
    width: int = 1     # boxcar width in samples
    dm: float = 0.0    # for bookkeeping / labels only


@dataclass
class Burst:
    t: int
    dur: int


@dataclass
class BeamRecipe:
    pulses: list = field(default_factory=list)
    stuck_channels: np.ndarray = field(default_factory=lambda: np.zeros(0, dtype=np.int64))
    bursts: list = field(default_factory=list)


def apply_recipe(levels: np.ndarray, recipe: BeamRecipe) -> np.ndarray:
    """Inject pulses, stuck channels and zero-DM bursts in place (clip at 3)."""
    nchan, nsamp = levels.shape
    for p in recipe.pulses:
        offs = np.asarray(p.offsets, dtype=np.int64)
        for c in range(nchan):
            a = p.t0 + int(offs[c])
            lo, hi = max(a, 0), min(a + p.width, nsamp)
            if lo < hi:
                seg = levels[c, lo:hi].astype(np.int16) + p.amp
                levels[c, lo:hi] = np.minimum(seg, 3).astype(np.uint8)
    for c in recipe.stuck_channels:
        levels[int(c), :] = 3
    for b in recipe.bursts:
        lo, hi = max(b.t, 0), min(b.t + b.dur, nsamp)
        if lo < hi:
            levels[:, lo:hi] = 3
    return levels


def draw_recipe(rng: np.random.Generator, nchan: int, nsamp_out: int, dm_max: float,
                offsets_for_dm, npulses: int = 20, dm_range=(5.0, 900.0), width_range=(1, 250),
                stuck_frac: float = 0.05, nbursts: int = 3, burst_range=(16, 781)) -> BeamRecipe:
    """Draw the multibeam injection recipe.

    offsets_for_dm(dm) -> int array [nchan] of per-channel arrival offsets; the
    caller decides how they are computed.
    """
    rec = BeamRecipe()
    hi_dm = min(dm_range[1], dm_max)
    for _ in range(npulses):
        dm = float(rng.uniform(dm_range[0], hi_dm))
        w = int(rng.integers(width_range[0], width_range[1] + 1))
        amp = int(rng.integers(1, 3))
        t0 = int(rng.integers(0, max(nsamp_out - w, 1)))
        rec.pulses.append(Pulse(t0=t0, offsets=np.asarray(offsets_for_dm(dm)), amp=amp, width=w, dm=dm))
    nstuck = int(round(stuck_frac * nchan))
    rec.stuck_channels = np.sort(rng.choice(nchan, size=nstuck, replace=False))
    for _ in range(nbursts):
        dur = int(rng.integers(burst_range[0], burst_range[1] + 1))
        t = int(rng.integers(0, max(nsamp_out - dur, 1)))
        rec.bursts.append(Burst(t=t, dur=dur))
    return rec


def make_gulp(seed: int, nchan: int, nsamp: int, recipe: BeamRecipe | None = None,
              ld_bytes: int | None = None, background: str = "noise"):
    """-> (packed uint8 [nchan, ld_bytes], levels uint8 [nchan, nsamp])."""
    rng = np.random.default_rng(seed)
    if background == "noise":
        lv = noise_levels(rng, nchan, nsamp)
    elif background == "zero":
        lv = np.zeros((nchan, nsamp), dtype=np.uint8)
    elif background == "max":
        lv = np.full((nchan, nsamp), 3, dtype=np.uint8)
    else:
        raise ValueError(background)
    if recipe is not None:
        apply_recipe(lv, recipe)
    return pack2(lv, ld_bytes), lv


# ---- device-side generation (large gulps) ------------------------------------

def device_noise_packed(nchan: int, nsamp: int, seed: int, device="cuda", ld_bytes: int | None = None):
    """Packed quantised noise generated with torch's seeded device RNG.

    Same distribution and packing as make_gulp(background="noise"); used where
    host generation of hundreds of MB per gulp would dominate.
    """
    import torch

    if ld_bytes is None:
        ld_bytes = padded_row_bytes(nsamp)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    out = torch.empty((nchan, ld_bytes), dtype=torch.uint8, device=device)
    cuts = [int(c) for c in _CUTS32]
    rows = max(1, (1 << 26) // max(ld_bytes * 4, 1))
    for c0 in range(0, nchan, rows):
        c1 = min(nchan, c0 + rows)
        u = torch.randint(0, 2**32, (c1 - c0, ld_bytes * 4), generator=g, device=device, dtype=torch.int64)
        lv = (u >= cuts[0]).to(torch.uint8) + (u >= cuts[1]).to(torch.uint8) + (u >= cuts[2]).to(torch.uint8)
        lv[:, nsamp:] = 0
        lv = lv.view(c1 - c0, ld_bytes, 4)
        out[c0:c1] = lv[:, :, 0] | (lv[:, :, 1] << 2) | (lv[:, :, 2] << 4) | (lv[:, :, 3] << 6)
    return out


def _device_or_levels(packed, c_idx, t_idx, fn):
    """Read-modify-write of individual 2-bit samples of a device gulp.

    c_idx, t_idx: int64 device tensors of distinct (channel, sample) pairs;
    fn maps the old levels (int16) to the new ones.  Samples sharing a byte are
    handled in four passes by t % 4 so no byte is written twice in a pass."""
    import torch

    ld = packed.shape[1]
    flat = packed.view(-1)
    for r in range(4):
        m = (t_idx % 4) == r
        if not bool(m.any()):
            continue
        bi = c_idx[m] * ld + t_idx[m] // 4
        old = flat[bi]
        lv = ((old >> (2 * r)) & 3).to(torch.int16)
        new = fn(lv).to(torch.uint8)
        flat[bi] = (old & ~(3 << (2 * r)) & 0xFF) | (new << (2 * r))


def device_apply_recipe(packed, nsamp: int, recipe: BeamRecipe):
    """Apply a recipe to a device-resident packed gulp: pulses add +amp with
    clipping at 3, stuck channels and zero-DM bursts are set to level 3."""
    import torch

    dev = packed.device
    nchan = packed.shape[0]
    chans = torch.arange(nchan, device=dev, dtype=torch.int64)
    for p in recipe.pulses:
        offs = torch.as_tensor(np.asarray(p.offsets, dtype=np.int64), device=dev)
        k = torch.arange(p.width, device=dev, dtype=torch.int64)
        t = (p.t0 + offs)[:, None] + k[None, :]
        c = chans[:, None].expand_as(t)
        ok = (t >= 0) & (t < nsamp)
        amp = int(p.amp)
        _device_or_levels(packed, c[ok], t[ok], lambda lv: torch.clamp(lv + amp, max=3))
    three = lambda lv: torch.full_like(lv, 3)
    if len(recipe.stuck_channels):
        idx = torch.as_tensor(np.asarray(recipe.stuck_channels, dtype=np.int64), device=dev)
        full = nsamp // 4
        packed[idx, :full] = 0xFF
        if nsamp % 4:
            tt = torch.arange(full * 4, nsamp, device=dev, dtype=torch.int64)
            cc = idx[:, None].expand(-1, tt.numel()).reshape(-1)
            _device_or_levels(packed, cc, tt.repeat(idx.numel()), three)
    for b in recipe.bursts:
        lo, hi = max(b.t, 0), min(b.t + b.dur, nsamp)
        if lo >= hi:
            continue
        a, z = (lo + 3) // 4, hi // 4
        if a < z:
            packed[:, a:z] = 0xFF
        edge = [t for t in range(lo, hi) if not (a * 4 <= t < z * 4)]
        if edge:
            tt = torch.as_tensor(edge, device=dev, dtype=torch.int64)
            cc = chans[:, None].expand(-1, tt.numel()).reshape(-1)
            _device_or_levels(packed, cc, tt.repeat(nchan), three)
    return packed
