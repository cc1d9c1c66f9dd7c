"""Host-side statistics of the classifier evaluation (no GPU): the Wilson
interval against scipy's binomial test, and the matched-recall counts against
a brute-force search over thresholds."""
import numpy as np
import pytest


def test_wilson_interval_matches_scipy():
    stats = pytest.importorskip("scipy.stats")
    from paper_1112_0065_gb300.training import wilson_interval

    for k, n in [(313, 323), (330, 350), (344, 432), (0, 10), (10, 10), (1, 2), (347, 408395)]:
        lo, hi = wilson_interval(k, n)
        ci = stats.binomtest(k, n).proportion_ci(confidence_level=0.95, method="wilson")
        assert abs(lo - ci.low) < 1e-9 and abs(hi - ci.high) < 1e-9, (k, n)


def test_matched_point_is_the_largest_threshold_reaching_the_recall():
    from paper_1112_0065_gb300.training import matched_point

    rng = np.random.default_rng(0)
    for _ in range(20):
        n = int(rng.integers(5, 60))
        scores = rng.integers(0, 15, n).astype(np.float64)     # ties included
        labels = (rng.random(n) < 0.3).astype(np.float32)
        if labels.sum() == 0:
            labels[0] = 1
        npos = int(labels.sum())
        for recall in (0.5, 0.9, 1.0):
            thr, sel, tp, pos = matched_point(scores, labels, recall)
            assert pos == npos and tp >= int(np.ceil(recall * npos))
            # brute force over the sorted order (stable, as the function ranks)
            order = np.argsort(-scores, kind="stable")
            best = None
            for k in range(1, n + 1):
                if labels[order[:k]].sum() >= np.ceil(recall * npos):
                    best = k
                    break
            assert sel == best and thr == scores[order[best - 1]]
            assert tp == int(labels[order[:best]].sum())
