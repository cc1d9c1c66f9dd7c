"""Train and evaluate the candidate classifier on pipeline candidates.

The data come from the GPU pipeline itself: synthetic 2-bit gulps of the
single-beam HTRU shape with injected dispersed pulses, stuck channels and
zero-DM bursts are dedispersed, searched (running-median baseline, boxcars
1..1024, S/N >= 6, grouping) and cut into 64x64 bfloat16 snippets.  A
candidate is labelled astrophysical when an injected pulse lies within 2 DM
trials of it (trial nearest the pulse's DM) and within the pulse's width in
time.  The classifier is compared with the plain S/N threshold at matched
recall.

  python -m paper_1112_0065_gb300.training --train-gulps 8 --eval-gulps 2 --out clf.ckpt
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

from . import _lib  # noqa: F401  (fails loudly without the native library)
from .classifier import Classifier
from .dedisp import Plan, compute_delays
from .search import DEFAULT_WIDTHS, Search

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if _ROOT not in sys.path:
    sys.path.insert(0, _ROOT)
import synth  # noqa: E402


class CandidateSource:
    """Runs dedispersion + search + snippets on synthetic gulps."""

    def __init__(self, nchan=1024, dm_max=1000.0, nout=1 << 19, half_window=4096, thresh=6.0,
                 max_cands=1 << 18, device="cuda"):
        self.f = synth.band_freqs(nchan)
        self.dms = synth.dm_list_piecewise(dm_max)
        self.plan = Plan(self.f, synth.TSAMP_HTRU, self.dms)
        self.nout = nout
        self.nsamp = nout + self.plan.maxdelay
        self.nchan = nchan
        self.dm_max = dm_max
        self.search = Search(len(self.dms), nout, nchan=nchan, half_window=half_window, widths=DEFAULT_WIDTHS,
                             thresh=thresh, max_cands=max_cands, full_map=False)
        self.out = self.plan.alloc_output(self.nsamp)
        self.device = device

    def offsets(self, dm):
        return compute_delays(self.f, synth.TSAMP_HTRU, [dm])[0]

    def gulp(self, seed, npulses=20, **recipe_kw):
        """-> (candidates structured array, snippets bf16 tensor [k,64,64], recipe)."""
        rng = np.random.default_rng(seed)
        rec = synth.draw_recipe(rng, self.nchan, self.nout, self.dm_max, self.offsets, npulses=npulses, **recipe_kw)
        d_in = synth.device_noise_packed(self.nchan, self.nsamp, seed=seed, device=self.device)
        synth.device_apply_recipe(d_in, self.nsamp, rec)
        self.plan.execute(d_in, self.nsamp, self.out)
        self.search.run(self.out, len(self.dms), self.nout)
        cands = self.search.candidates()
        snips = self.search.snippets(len(cands))
        return cands, snips.clone(), rec

    def labels(self, cands, rec, dm_tol=2):
        lab = np.zeros(len(cands), dtype=np.float32)
        for p in rec.pulses:
            dp = int(np.argmin(np.abs(self.dms - p.dm)))
            hit = (np.abs(cands["d"] - dp) <= dm_tol) & (np.abs(cands["t"] - p.t0) <= p.width)
            lab[hit] = 1.0
        return lab

    def close(self):
        self.search.close()
        self.plan.close()


def precision_at_recall(scores, labels, recall):
    """Precision of `score >= thr` with thr the largest threshold reaching the recall."""
    pos = labels > 0.5
    npos = int(pos.sum())
    if npos == 0:
        return float("nan"), float("nan")
    order = np.argsort(-scores, kind="stable")
    tp = np.cumsum(pos[order])
    k = int(np.searchsorted(tp, int(np.ceil(recall * npos))))
    k = min(k, len(order) - 1)
    return float(tp[k] / (k + 1)), float(scores[order[k]])


def train(clf, x, y, steps, batch=256, lr=2e-3, seed=0, balance=True, log_every=0):
    """Mini-batch AdamW with class-balanced sampling (positives are rare)."""
    import torch

    rng = np.random.default_rng(seed)
    pos = np.flatnonzero(y > 0.5)
    neg = np.flatnonzero(y <= 0.5)
    yd = torch.from_numpy(y).to(x.device)
    losses = []
    for s in range(steps):
        if balance and len(pos) and len(neg):
            idx = np.concatenate([rng.choice(pos, batch // 2), rng.choice(neg, batch - batch // 2)])
        else:
            idx = rng.choice(len(y), batch)
        it = torch.from_numpy(idx).to(x.device)
        lr_s = lr * 0.5 * (1 + np.cos(np.pi * s / max(steps, 1)))  # cosine schedule
        clf.train_step(x.index_select(0, it).contiguous(), yd.index_select(0, it).contiguous(), lr=float(lr_s))
        if log_every and (s % log_every == 0 or s == steps - 1):
            losses.append((s, clf.loss()))
    return losses


def score(clf, x, batch=1024):
    import torch

    out = []
    for i in range(0, x.shape[0], batch):
        out.append(clf.forward(x[i:i + batch].contiguous()).clone())
    torch.cuda.synchronize()
    return torch.cat(out).cpu().numpy() if out else np.zeros(0, np.float32)


def run(train_gulps=8, eval_gulps=2, train_pulses=100, eval_pulses=20, steps=1500, batch=256, lr=2e-3, nout=1 << 19,
        seed=synth.BASE_SEED + 4000, out=None, log=print):
    import torch

    src = CandidateSource(nout=nout)
    xs, ys, snrs = [], [], []
    t0 = time.time()
    for g in range(train_gulps):
        c, sn, rec = src.gulp(seed + g, npulses=train_pulses)
        xs.append(sn)
        ys.append(src.labels(c, rec))
        snrs.append(c["snr"])
    x = torch.cat(xs)
    y = np.concatenate(ys)
    t_data = time.time() - t0
    log(f"train candidates: {len(y)} ({int(y.sum())} astrophysical) from {train_gulps} gulps in {t_data:.1f} s")
    clf = Classifier(max_batch=max(batch, 1024), seed=seed)
    t0 = time.time()
    losses = train(clf, x, y, steps, batch=batch, lr=lr, seed=seed, log_every=max(steps // 10, 1))
    torch.cuda.synchronize()
    t_train = time.time() - t0
    log(f"trained {steps} steps x {batch} in {t_train:.1f} s; loss {losses[0][1]:.4f} -> {losses[-1][1]:.4f}")
    del x, xs
    ex, ey, esnr = [], [], []
    for g in range(eval_gulps):
        c, sn, rec = src.gulp(seed + 1000 + g, npulses=eval_pulses)
        ex.append(score(clf, sn))
        ey.append(src.labels(c, rec))
        esnr.append(c["snr"])
    z = np.concatenate(ex)
    yv = np.concatenate(ey)
    sv = np.concatenate(esnr)
    rep = {"train_candidates": int(len(y)), "train_positives": int(y.sum()), "eval_candidates": int(len(yv)),
           "eval_positives": int(yv.sum()), "steps": steps, "batch": batch, "train_s": round(t_train, 2),
           "data_s": round(t_data, 2), "loss_first": losses[0][1], "loss_last": losses[-1][1],
           "snr6_precision": float(yv.mean()) if len(yv) else float("nan"), "matched": []}
    for r in (0.9, 0.95, 0.99, 1.0):
        pc, thr_c = precision_at_recall(z, yv, r)
        ps, thr_s = precision_at_recall(sv, yv, r)
        rep["matched"].append({"recall": r, "classifier_precision": pc, "snr_precision": ps,
                               "classifier_logit_thr": thr_c, "snr_thr": thr_s})
    if out:
        clf.save(out)
    src.close()
    clf.close()
    return rep


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train-gulps", type=int, default=8)
    ap.add_argument("--eval-gulps", type=int, default=2)
    ap.add_argument("--train-pulses", type=int, default=100)
    ap.add_argument("--steps", type=int, default=1500)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--nout-log2", type=int, default=19)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    rep = run(a.train_gulps, a.eval_gulps, a.train_pulses, 20, a.steps, a.batch, a.lr, 1 << a.nout_log2, out=a.out)
    print(json.dumps(rep))


if __name__ == "__main__":
    main()
