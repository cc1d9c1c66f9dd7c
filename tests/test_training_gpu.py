"""End-to-end learned stage: candidates produced by the GPU pipeline from
synthetic gulps (dispersed pulses, stuck channels, zero-DM bursts), labelled
by injection match, train the classifier with its own GPU kernels; on
held-out gulps it ranks candidates better than the plain S/N threshold."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_precision_at_recall_definition():
    from paper_1112_0065_gb300.training import precision_at_recall

    s = np.array([9.0, 8.0, 7.0, 6.0, 5.0])
    y = np.array([1, 0, 1, 0, 1], dtype=np.float32)
    assert precision_at_recall(s, y, 1 / 3)[0] == 1.0
    assert abs(precision_at_recall(s, y, 2 / 3)[0] - 2 / 3) < 1e-12
    assert abs(precision_at_recall(s, y, 1.0)[0] - 3 / 5) < 1e-12


def test_classifier_beats_snr_threshold_at_matched_recall():
    from paper_1112_0065_gb300 import training

    rep = training.run(train_gulps=6, eval_gulps=3, train_pulses=60, eval_pulses=40, steps=600, batch=128,
                       nout=1 << 18, log=lambda *a: None)
    assert rep["eval_positives"] >= 30 and rep["train_positives"] >= 100
    assert rep["loss_last"] < 0.1 * rep["loss_first"]
    gains = [m["classifier_precision"] - m["snr_precision"] for m in rep["matched"] if m["recall"] <= 0.95]
    assert min(gains) >= 0.0 and max(gains) > 0.0, rep["matched"]
