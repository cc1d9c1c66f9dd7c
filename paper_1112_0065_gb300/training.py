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
  python -m paper_1112_0065_gb300.training --report PATH     # held-out evaluation against the S/N cut
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


def wilson_interval(k: int, n: int, z: float = 1.959963984540054):
    """Wilson score interval (95 % by default) of a binomial proportion k/n."""
    if n <= 0:
        return float("nan"), float("nan")
    p = k / n
    den = 1.0 + z * z / n
    centre = (p + z * z / (2 * n)) / den
    half = z * np.sqrt(p * (1 - p) / n + z * z / (4.0 * n * n)) / den
    return float(centre - half), float(centre + half)


def matched_point(scores, labels, recall):
    """Counts at the largest threshold whose `score >= thr` reaches `recall`:
    (threshold, selected, true positives, positives)."""
    pos = labels > 0.5
    npos = int(pos.sum())
    order = np.argsort(-scores, kind="stable")
    tp = np.cumsum(pos[order])
    k = min(int(np.searchsorted(tp, int(np.ceil(recall * npos)))), len(order) - 1)
    return float(scores[order[k]]), k + 1, int(tp[k]), npos


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


def evaluate(train_candidates=200_000, train_positives=1000, max_train_gulps=40, eval_gulps=12, train_pulses=100,
             eval_pulses=50, steps=6000, batch=256, lr=2e-3, nout=1 << 19, seed=synth.BASE_SEED + 6000, log=print):
    """The learned classifier against the plain S/N threshold on held-out
    gulps, at matched recall, with counts and 95 % Wilson intervals.

    Training gulps (seeds seed, seed+1, ...) are generated until at least
    `train_candidates` pipeline candidates, `train_positives` of them
    astrophysical, exist (at most `max_train_gulps`); evaluation gulps use
    seeds from seed+10000 on, none shared with training.  Both the fixed-order
    forward (the served path) and the tensor-core forward score the
    evaluation set; their decisions are compared at every matched threshold.
    """
    import torch

    src = CandidateSource(nout=nout)
    xs, ys = [], []
    t0 = time.time()
    ntr, npos, g = 0, 0, 0
    while (ntr < train_candidates or npos < train_positives) and g < max_train_gulps:
        c, sn, rec = src.gulp(seed + g, npulses=train_pulses)
        xs.append(sn)
        ys.append(src.labels(c, rec))
        ntr += len(c)
        npos += int(ys[-1].sum())
        g += 1
    x = torch.cat(xs)
    y = np.concatenate(ys)
    del xs
    t_data = time.time() - t0
    log(f"train: {len(y)} candidates ({int(y.sum())} astrophysical) from {g} gulps in {t_data:.1f} s")
    clf = Classifier(max_batch=max(batch, 8192), seed=seed)
    t0 = time.time()
    losses = train(clf, x, y, steps, batch=batch, lr=lr, seed=seed, log_every=max(steps // 10, 1))
    torch.cuda.synchronize()
    t_train = time.time() - t0
    log(f"trained {steps} x {batch} in {t_train:.1f} s; loss {losses[0][1]:.4f} -> {losses[-1][1]:.4f}")
    del x
    z, ztc, yv, sv, per_gulp = [], [], [], [], []
    for k in range(eval_gulps):
        c, sn, rec = src.gulp(seed + 10000 + k, npulses=eval_pulses)
        z.append(score(clf, sn, batch=8192))
        out = []
        for i in range(0, sn.shape[0], 8192):
            out.append(clf.forward(sn[i:i + 8192].contiguous(), tensor_cores=True).clone())
        torch.cuda.synchronize()
        ztc.append(torch.cat(out).cpu().numpy() if out else np.zeros(0, np.float32))
        lab = src.labels(c, rec)
        yv.append(lab)
        sv.append(c["snr"])
        per_gulp.append({"candidates": int(len(c)), "positives": int(lab.sum()), "pulses": len(rec.pulses)})
    z, ztc, yv, sv = (np.concatenate(a) for a in (z, ztc, yv, sv))
    tc_status = clf.status()
    rep = {"train_gulps": g, "train_candidates": int(len(y)), "train_positives": int(y.sum()),
           "eval_gulps": eval_gulps, "eval_candidates": int(len(yv)), "eval_positives": int(yv.sum()),
           "eval_per_gulp": per_gulp, "train_pulses_per_gulp": train_pulses, "eval_pulses_per_gulp": eval_pulses,
           "steps": steps, "batch": batch, "lr": lr, "seeds": {"train_first": seed, "eval_first": seed + 10000},
           "train_s": round(t_train, 2), "data_s": round(t_data, 2),
           "loss_first": round(losses[0][1], 5), "loss_last": round(losses[-1][1], 5),
           "snr6_precision": float(yv.mean()), "matched": [],
           "tensor_cores": {"status": int(tc_status), "max_abs_logit_diff": float(np.max(np.abs(z - ztc))),
                            "frac_within_1e-3": float(np.mean(np.abs(z - ztc) <= 1e-3))}}
    for r in (0.9, 0.95, 0.99):
        row = {"recall": r}
        for name, sc in (("classifier", z), ("snr", sv)):
            thr, sel, tp, npos = matched_point(sc, yv, r)
            lo, hi = wilson_interval(tp, sel)
            row[name] = {"threshold": round(thr, 5), "selected": sel, "true_positives": tp, "positives": npos,
                         "recall": round(tp / npos, 5), "precision": round(tp / sel, 5),
                         "precision_ci95": [round(lo, 5), round(hi, 5)]}
        thr = row["classifier"]["threshold"]
        agree = float(np.mean((z >= thr) == (ztc >= thr)))
        sel_tc = ztc >= thr
        tp_tc = int((sel_tc & (yv > 0.5)).sum())
        row["tensor_cores_at_classifier_threshold"] = {
            "decision_agreement": round(agree, 6), "selected": int(sel_tc.sum()), "true_positives": tp_tc,
            "precision": round(tp_tc / max(int(sel_tc.sum()), 1), 5)}
        rep["matched"].append(row)
    sel0 = z >= 0.0
    tp0 = int((sel0 & (yv > 0.5)).sum())
    rep["classifier_at_logit0"] = {"selected": int(sel0.sum()), "true_positives": tp0,
                                   "recall": round(tp0 / max(int(yv.sum()), 1), 5),
                                   "precision": round(tp0 / max(int(sel0.sum()), 1), 5)}
    src.close()
    clf.close()
    return rep


def report_markdown(rep) -> str:
    """A short markdown summary of an evaluate() report."""
    lines = ["# Learned classifier against the plain S/N threshold, single HTRU-shaped beam", "",
             "1024 channels x 1500 DM trials x 2^19-sample gulps with dispersed pulses, 5 % stuck channels and 3 "
             "zero-DM bursts each, searched by the library (median baseline, boxcars 1..1024, S/N >= 6, grouping); "
             "a candidate is astrophysical when an injected pulse lies within 2 trials and its width of it.  "
             "Made by `python -m paper_1112_0065_gb300.training --report <path>` on one GB300.", "",
             f"Training: {rep['train_candidates']} pipeline candidates ({rep['train_positives']} astrophysical) "
             f"from {rep['train_gulps']} gulps; {rep['steps']} AdamW steps of {rep['batch']} (class-balanced), "
             f"loss {rep['loss_first']} -> {rep['loss_last']}.",
             f"Evaluation: {rep['eval_candidates']} candidates ({rep['eval_positives']} astrophysical) from "
             f"{rep['eval_gulps']} held-out gulps; the S/N >= 6 cut alone has precision "
             f"{rep['snr6_precision']:.4f} at recall 1.", "",
             "| recall | classifier precision (95 % CI) | selected / true | S/N precision (95 % CI) | selected / true "
             "| tensor-core decisions agreeing |", "|---|---|---|---|---|---|"]
    for m in rep["matched"]:
        c, s, t = m["classifier"], m["snr"], m["tensor_cores_at_classifier_threshold"]
        lines.append(f"| {m['recall']} | {c['precision']:.4f} ({c['precision_ci95'][0]:.4f}-{c['precision_ci95'][1]:.4f}) "
                     f"| {c['selected']} / {c['true_positives']} | {s['precision']:.4f} "
                     f"({s['precision_ci95'][0]:.4f}-{s['precision_ci95'][1]:.4f}) | {s['selected']} / "
                     f"{s['true_positives']} | {t['decision_agreement']:.6f} |")
    tc = rep["tensor_cores"]
    lines += ["", f"Tensor-core forward on the same set: max |logit difference| {tc['max_abs_logit_diff']:.4g}, "
              f"{100 * tc['frac_within_1e-3']:.2f} % of logits within 1e-3 (status {tc['status']})."]
    return "\n".join(lines) + "\n"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--report", metavar="PATH",
                    help="run the held-out evaluation against the S/N threshold and write PATH.json and PATH.md")
    ap.add_argument("--eval-gulps-report", type=int, default=12)
    ap.add_argument("--report-steps", type=int, default=6000)
    ap.add_argument("--eval-pulses", type=int, default=50)
    ap.add_argument("--train-gulps", type=int, default=8)
    ap.add_argument("--eval-gulps", type=int, default=2)
    ap.add_argument("--train-pulses", type=int, default=100)
    ap.add_argument("--steps", type=int, default=1500)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--nout-log2", type=int, default=19)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    if a.report:
        rep = evaluate(eval_gulps=a.eval_gulps_report, eval_pulses=a.eval_pulses, steps=a.report_steps,
                       batch=a.batch, lr=a.lr)
        with open(a.report + ".json", "w") as fh:
            json.dump(rep, fh, indent=1)
        with open(a.report + ".md", "w") as fh:
            fh.write(report_markdown(rep))
        print(report_markdown(rep))
        return
    rep = run(a.train_gulps, a.eval_gulps, a.train_pulses, 20, a.steps, a.batch, a.lr, 1 << a.nout_log2, out=a.out)
    print(json.dumps(rep))


if __name__ == "__main__":
    main()
