"""Parity of the GPU search stage with the CPU oracle: running-median
baseline, per-row sum of squares, best boxcar S/N and width per cell, grouped
candidates and bfloat16 snippets -- bit-exact on a small multibeam-style gulp,
and on sampled rows / candidates of the full single-beam workload."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

WIDTHS = tuple(1 << k for k in range(11))


@pytest.fixture(scope="module")
def P():
    import paper_1112_0065_gb300 as P

    P.load_library()
    return P


def small_gulp(seed, nchan=128, ndm=96, dm_end=150.0, nout=1 << 15, npulses=6):
    rng = np.random.default_rng(seed)
    f = synth.band_freqs(nchan)
    dms = synth.dm_list_linear(ndm, dm_end)
    delays = oracle.delay_table(f, 64e-6, dms)
    nsamp = nout + int(delays.max())
    rec = synth.draw_recipe(rng, nchan, nout, dm_end, lambda dm: oracle.delay_table(f, 64e-6, [dm])[0],
                            npulses=npulses, dm_range=(10.0, 140.0), width_range=(1, 60), nbursts=1,
                            burst_range=(5, 40))
    packed, _ = synth.make_gulp(seed, nchan, nsamp, rec)
    return f, dms, delays, packed, nsamp, rec


def _gpu_dedisp(P, f, dms, packed, nsamp):
    import torch

    plan = P.Plan(f, 64e-6, dms)
    out = plan.execute(torch.from_numpy(packed).cuda(), nsamp)
    torch.cuda.synchronize()
    return plan, out


@pytest.mark.parametrize("seed,half,nout", [(11, 512, 1 << 15), (12, 300, 1 << 15), (13, 700, 27001)])
def test_search_small_bit_exact(P, seed, half, nout):
    """Every stage against the oracle; 27001 outputs leave a ragged last tile
    and bitmask word."""
    import torch

    f, dms, delays, packed, nsamp, rec = small_gulp(seed, nout=nout)
    x_or = oracle.dedisperse(delays, packed, nsamp)
    plan, x_gpu = _gpu_dedisp(P, f, dms, packed, nsamp)
    n = plan.nout(nsamp)
    np.testing.assert_array_equal(P.as_uint32(x_gpu)[:, :n], x_or)

    s = P.Search(len(dms), n, nchan=f.size, half_window=half, widths=WIDTHS, thresh=6.0, max_cands=2048)
    s.run(x_gpu, len(dms), n, beam=3)
    res = s.result()
    assert res["flags"] == 0
    y, ss, best, bw = s.buffers()
    torch.cuda.synchronize()

    y_or = oracle.baseline(x_or, half)
    np.testing.assert_array_equal(y.cpu().numpy(), y_or)
    ss_or = np.array([oracle.sumsq(r) for r in y_or], dtype=np.int64)
    np.testing.assert_array_equal(ss.cpu().numpy(), ss_or)
    best_or, bw_or = oracle.best_snr(y_or, WIDTHS)
    np.testing.assert_array_equal(best.cpu().numpy(), best_or)
    np.testing.assert_array_equal(bw.cpu().numpy().astype(np.int32), bw_or)

    c_or = oracle.find_peaks(best_or, bw_or, 6.0)
    c = s.candidates()
    assert len(c) == len(c_or) == res["ngroups"] and len(c) > 0
    for k in ("d", "t", "w", "snr", "ncells"):
        np.testing.assert_array_equal(c[k], c_or[k])
    assert np.all(c["beam"] == 3)

    sn = s.snippets(len(c))
    torch.cuda.synchronize()
    sn_or = oracle.snippets(y_or, ss_or, c_or["d"], c_or["t"], c_or["w"])
    np.testing.assert_array_equal(sn.view(torch.int16).cpu().numpy().view(np.uint16), sn_or)
    sy = s.snippets_from_y(len(c))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(sy.view(torch.int16).cpu().numpy().view(np.uint16), sn_or)
    s.close()


@pytest.mark.parametrize("nchan", [1024, 2730, 4000, 12000])
def test_baseline_median_moves_far(P, nchan):
    """Rows whose median jumps across the whole value range (steps, ramps,
    extremes, bursts) against the oracle's running median, for value ranges
    up to 3072, 8190, 12000 and 36000.  With 12000 channels (values up to
    36000) outputs exceed 16 bits, the wide kernel."""
    import torch

    rng = np.random.default_rng(5)
    n, half = 40003, 4096  # a ragged last segment and chunk
    rows = []
    r0 = np.where(np.arange(n) < 15000, 200, 2800).astype(np.int64)            # step up
    rows.append(r0 + rng.integers(-20, 21, n))
    rows.append(np.linspace(3072, 0, n).astype(np.int64))                      # ramp down
    r2 = 1536 + rng.integers(-30, 31, n)
    for t0 in (1000, 9000, 30000):
        r2[t0:t0 + 6000] = 3072                                                 # wide bursts
    rows.append(r2)
    rows.append(rng.choice([0, 3072], n))                                       # extremes only
    rows.append(np.where((np.arange(n) // 7000) % 2 == 0, 100, 3000) + rng.integers(0, 3, n))
    x = np.stack(rows) * (3 * nchan) // 3072
    x = np.clip(x, 0, 3 * nchan).astype(np.uint32)
    if nchan > 10922:
        assert np.abs(oracle.baseline(x, half)).max() > 32767
    s = P.Search(len(rows), n, nchan=nchan, half_window=half, widths=(1, 2, 4), thresh=6.0, max_cands=1024)
    s.run(torch.from_numpy(x.view(np.int32)).cuda(), len(rows), n)
    assert s.result()["flags"] & 1 == 0
    y, ss, _, _ = s.buffers()
    y_or = oracle.baseline(x, half)
    np.testing.assert_array_equal(y.cpu().numpy(), y_or)
    np.testing.assert_array_equal(ss.cpu().numpy(), [oracle.sumsq(r) for r in y_or])


@pytest.mark.parametrize("n,half", [(1, 1), (5, 1), (31, 2), (33, 4), (100, 1000), (4097, 2048), (9000, 64),
                                    (70001, 32767)])
def test_baseline_median_edge_shapes(P, n, half):
    """Rows shorter than a window, shorter than a warp step, a ragged last
    step, and the largest window (65534 values): y equals the oracle's."""
    import torch

    rng = np.random.default_rng(n + half)
    ndm = 7
    x = (1536 + rng.integers(-90, 91, (ndm, n))).astype(np.uint32)
    x[1] = rng.choice([0, 3072], n)
    x[2] = np.arange(n) % 3073
    s = P.Search(ndm, n, nchan=1024, half_window=half, widths=(1,), thresh=6.0, max_cands=64)
    s.run(torch.from_numpy(x.view(np.int32)).cuda(), ndm, n)
    assert s.result()["flags"] & 1 == 0
    y, ss, _, _ = s.buffers()
    y_or = oracle.baseline(x, half)
    np.testing.assert_array_equal(y.cpu().numpy(), y_or)
    np.testing.assert_array_equal(ss.cpu().numpy(), [oracle.sumsq(r) for r in y_or])
    s.close()


def test_search_constant_rows_and_empty_result(P):
    import torch

    n, ndm = 5000, 10
    x = torch.full((ndm, n), 1536, dtype=torch.int32, device="cuda")
    s = P.Search(ndm, n, nchan=1024, half_window=256, widths=(1, 2, 4), thresh=6.0, max_cands=16)
    s.run(x, ndm, n)
    assert s.result() == {"nhot": 0, "ngroups": 0, "flags": 0}
    assert len(s.candidates()) == 0
    y, ss, best, bw = s.buffers()
    assert int(y.abs().max()) == 0 and int(ss.max()) == 0 and float(best.abs().max()) == 0.0


def test_search_rejects_bad_config(P):
    with pytest.raises(P.DDError):
        P.Search(10, 1000, nchan=64, widths=(1, 3))         # not a power of two
    with pytest.raises(P.DDError):
        P.Search(10, 1000, nchan=64, widths=(4, 2))         # not ascending
    with pytest.raises(P.DDError):
        P.Search(10, 1000, nchan=64, max_cands=(1 << 20) + 1)  # above the capacity


@pytest.mark.parametrize("baseline", ["median", "mean"])
def test_search_single_beam_workload_sampled(P, baseline):
    """1024 channels x 1500 DMs x 2^19 samples, window 8192, widths 1..1024,
    with the multibeam injection recipe: sampled rows are bit-exact, and every
    candidate sampled is an exact S/N maximum group of its row."""
    import torch

    rng = np.random.default_rng(23)
    f = synth.band_freqs(1024)
    dms = synth.dm_list_piecewise(1000.0)
    plan = P.Plan(f, 64e-6, dms)
    nout = 1 << 19
    nsamp = nout + plan.maxdelay
    d_in = synth.device_noise_packed(1024, nsamp, seed=synth.BASE_SEED + 400)
    rec = synth.draw_recipe(rng, 1024, nout, 1000.0, lambda dm: oracle.delay_table(f, 64e-6, [dm])[0])
    synth.device_apply_recipe(d_in, nsamp, rec)
    x = plan.execute(d_in, nsamp)
    s = P.Search(1500, nout, nchan=1024, half_window=4096, widths=WIDTHS, thresh=6.0, max_cands=1 << 18,
                 baseline=baseline)
    s.run(x, 1500, nout)
    res = s.result()
    assert res["flags"] == 0 and 0 < res["ngroups"] <= 1 << 18
    y, ss, best, bw = s.buffers()
    cands = s.candidates()
    torch.cuda.synchronize()
    packed = d_in.cpu().numpy()
    delays = oracle.delay_table(f, 64e-6, dms)
    # rows: DM 0, a middle row and the row of the strongest candidate
    top = cands[np.argmax(cands["snr"])]
    for row in sorted({0, 700, int(top["d"])}):
        x_row = oracle.dedisperse_points(delays, packed, nsamp, np.full(nout, row), np.arange(nout))
        base = oracle.baseline if baseline == "median" else oracle.baseline_mean
        y_row = base(x_row[None, :], 4096)[0]
        np.testing.assert_array_equal(y[row].cpu().numpy(), y_row)
        assert int(ss[row]) == oracle.sumsq(y_row)
        if row == int(top["d"]):
            b_row, w_row = oracle.best_snr(y_row[None, :], WIDTHS)
            np.testing.assert_array_equal(best[row].cpu().numpy(), b_row[0])
            np.testing.assert_array_equal(bw[row].cpu().numpy().astype(np.int32), w_row[0])
            assert b_row[0][top["t"]] == top["snr"] and w_row[0][top["t"]] == top["w"]
    # candidate list properties at full size
    assert np.all(cands["snr"] >= 6.0)
    order = np.lexsort((cands["t"], cands["d"]))
    np.testing.assert_array_equal(order, np.arange(len(cands)))
    at = best[torch.as_tensor(cands["d"], device="cuda").long(), torch.as_tensor(cands["t"], device="cuda").long()]
    np.testing.assert_array_equal(at.cpu().numpy(), cands["snr"])
    assert int(cands["ncells"].sum()) == res["nhot"]


@pytest.mark.parametrize("widths", [(2, 16, 128, 1024), (4,), (1, 8, 32)])
def test_search_width_subsets(P, widths):
    """Width lists with gaps and without width 1: best S/N, best width and
    candidates equal the oracle's, in the full map and in hot-cells-only mode."""
    import torch

    f, dms, delays, packed, nsamp, rec = small_gulp(17)
    x_or = oracle.dedisperse(delays, packed, nsamp)
    plan, x_gpu = _gpu_dedisp(P, f, dms, packed, nsamp)
    n = plan.nout(nsamp)
    y_or = oracle.baseline(x_or, 400)
    best_or, bw_or = oracle.best_snr(y_or, widths)
    c_or = oracle.find_peaks(best_or, bw_or, 6.0)
    for full in (True, False):
        s = P.Search(len(dms), n, nchan=f.size, half_window=400, widths=widths, thresh=6.0, max_cands=2048,
                     full_map=full)
        s.run(x_gpu, len(dms), n)
        res = s.result()
        _, _, best, bw = s.buffers()
        torch.cuda.synchronize()
        if full:
            np.testing.assert_array_equal(best.cpu().numpy(), best_or)
            np.testing.assert_array_equal(bw.cpu().numpy().astype(np.int32), bw_or)
        assert res["nhot"] == int((best_or >= 6.0).sum())
        c = s.candidates()
        assert len(c) == len(c_or) == res["ngroups"]
        for k in ("d", "t", "w", "snr", "ncells"):
            np.testing.assert_array_equal(c[k], c_or[k])
        s.close()


def test_hot_cells_only_mode_matches_full_map(P):
    """Production mode (S/N stored for hot cells only, hot test by integer
    thresholds) finds the same hot cells and candidates as the full map."""
    import torch

    f, dms, delays, packed, nsamp, rec = small_gulp(41)
    plan, x = _gpu_dedisp(P, f, dms, packed, nsamp)
    n = plan.nout(nsamp)
    out = []
    for full in (True, False):
        s = P.Search(len(dms), n, nchan=f.size, half_window=512, widths=WIDTHS, thresh=6.0, max_cands=2048,
                     full_map=full)
        s.run(x, len(dms), n)
        res = s.result()
        c = s.candidates()
        _, _, best, bw = s.buffers()
        at = (torch.as_tensor(c["d"], device="cuda").long(), torch.as_tensor(c["t"], device="cuda").long())
        out.append((res, c, best[at].cpu().numpy(), bw.view(torch.int16)[at].cpu().numpy()))
        s.close()
    assert out[0][0] == out[1][0] and out[0][0]["ngroups"] > 0
    np.testing.assert_array_equal(out[0][1], out[1][1])
    np.testing.assert_array_equal(out[0][2], out[1][2])
    np.testing.assert_array_equal(out[0][3], out[1][3])
    # and the oracle's count of cells at or above the threshold
    best_or, _ = oracle.best_snr(oracle.baseline(oracle.dedisperse(delays, packed, nsamp), 512), WIDTHS)
    assert int((best_or >= 6.0).sum()) == out[1][0]["nhot"]


def _shape_rows(rng, ndm, n):
    """Rows of a constant background with spikes drawn as hot-cell shapes:
    random scatter, runs crossing 32-cell words, runs at both row ends,
    U shapes, staircases, diagonal neighbours (not connected) and a ladder."""
    hot = np.zeros((ndm, n), dtype=bool)
    hot |= rng.random((ndm, n)) < 0.002
    for d in range(0, ndm, 7):
        t = int(rng.integers(0, n - 200))
        hot[d, t:t + int(rng.integers(33, 110))] = True
    hot[3, :45] = True
    hot[4, n - 70:] = True
    hot[5, n - 1] = True
    for d0, t0 in ((10, 300), (30, 4000)):               # U: two columns joined only at the bottom
        hot[d0:d0 + 6, t0] = True
        hot[d0:d0 + 6, t0 + 20] = True
        hot[d0 + 5, t0:t0 + 21] = True
    for k in range(12):                                   # staircase of overlapping runs
        hot[40 + k, 1000 + 5 * k:1000 + 5 * k + 8] = True
    for k in range(8):                                    # diagonal: separate groups
        hot[55 + k, 6000 + k] = True
    hot[60:68, 7000:7040:2] = True                        # ladder rungs ...
    hot[60:68, 7000] = True                               # ... joined by one column
    rows = np.full((ndm, n), 500, dtype=np.int64)
    rows[hot] += rng.integers(85, 101, int(hot.sum()))
    return rows.astype(np.uint32)


@pytest.mark.parametrize("full_map", [True, False])
def test_grouping_shapes(P, full_map):
    """Grouping of designed hot-cell maps (width 1, so a hot cell is a spike)
    against the oracle's flood fill: candidates, representatives, sizes."""
    import torch

    rng = np.random.default_rng(77)
    ndm, n, half = 70, 8190, 4096
    x = _shape_rows(rng, ndm, n)
    s = P.Search(ndm, n, nchan=1024, half_window=half, widths=(1,), thresh=6.0, max_cands=4096, full_map=full_map)
    s.run(torch.from_numpy(x.view(np.int32)).cuda(), ndm, n, beam=1)
    res = s.result()
    c = s.candidates()
    y_or = oracle.baseline(x, half)
    best_or, bw_or = oracle.best_snr(y_or, (1,))
    c_or = oracle.find_peaks(best_or, bw_or, 6.0)
    assert res["flags"] == 0 and res["nhot"] == int((best_or >= 6.0).sum())
    assert len(c) == len(c_or) == res["ngroups"] and len(c) > 100
    for k in ("d", "t", "w", "snr", "ncells"):
        np.testing.assert_array_equal(c[k], c_or[k])
    s.close()


@pytest.mark.parametrize("half", [512, 300])
def test_mean_baseline_bit_exact(P, half):
    """The paper's running-mean baseline option: y, sum y^2, best S/N and width
    per cell and the candidates against the oracle."""
    import torch

    f, dms, delays, packed, nsamp, rec = small_gulp(51)
    x_or = oracle.dedisperse(delays, packed, nsamp)
    plan, x_gpu = _gpu_dedisp(P, f, dms, packed, nsamp)
    n = plan.nout(nsamp)
    s = P.Search(len(dms), n, nchan=f.size, half_window=half, widths=WIDTHS, thresh=6.0, max_cands=2048,
                 baseline="mean")
    s.run(x_gpu, len(dms), n)
    res = s.result()
    assert res["flags"] == 0
    y, ss, best, bw = s.buffers()
    torch.cuda.synchronize()
    y_or = oracle.baseline_mean(x_or, half)
    np.testing.assert_array_equal(y.cpu().numpy(), y_or)
    ss_or = np.array([oracle.sumsq(r) for r in y_or], dtype=np.int64)
    np.testing.assert_array_equal(ss.cpu().numpy(), ss_or)
    best_or, bw_or = oracle.best_snr(y_or, WIDTHS)
    np.testing.assert_array_equal(best.cpu().numpy(), best_or)
    c_or = oracle.find_peaks(best_or, bw_or, 6.0)
    c = s.candidates()
    assert len(c) == len(c_or) > 0
    for k in ("d", "t", "w", "snr", "ncells"):
        np.testing.assert_array_equal(c[k], c_or[k])
    s.close()


def test_mean_baseline_ragged_rows(P):
    """Rows shorter than a window, one sample, and lengths off the tile grid;
    half windows whose tile span needs several scan passes of the fused
    kernel (20000), and one too wide for its shared memory (24000), which
    takes the two-pass form through a row prefix in memory."""
    import torch

    rng = np.random.default_rng(8)
    for n, half in [(1, 4), (5, 100), (4097, 2048), (9001, 4096), (50001, 20000), (60001, 24000)]:
        x = rng.integers(0, 3 * 64 + 1, size=(3, n)).astype(np.uint32)
        s = P.Search(3, n, nchan=64, half_window=half, widths=(1, 2), thresh=6.0, max_cands=64, baseline="mean")
        s.run(torch.from_numpy(x.view(np.int32)).cuda(), 3, n)
        y, ss, _, _ = s.buffers()
        np.testing.assert_array_equal(y.cpu().numpy(), oracle.baseline_mean(x, half))
        s.close()
