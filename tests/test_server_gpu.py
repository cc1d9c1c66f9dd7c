"""Streaming server: dedispersed outputs carried across gulps equal the
oracle's one-shot result over the concatenated stream; a beam's results are
the same alone and mixed with other beams' gulps in flight; admission refuses
work when no slot or device memory is free; bad submissions are rejected."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_1112_0065_gb300 as P

    P.load_library()
    return P


def stream_levels(seed, nchan, ngulps, G, with_pulses=True):
    rng = np.random.default_rng(seed)
    lv = synth.noise_levels(rng, nchan, ngulps * G)
    if with_pulses:
        f = synth.band_freqs(nchan)
        for k in range(3):
            dm = float(rng.uniform(5, 50))
            rec = synth.BeamRecipe(pulses=[synth.Pulse(t0=int(rng.integers(0, ngulps * G - 3000)),
                                                       offsets=oracle.delay_table(f, 64e-6, [dm])[0], amp=2,
                                                       width=int(rng.integers(1, 20)), dm=dm)])
            synth.apply_recipe(lv, rec)
    return lv


def gulp_bytes(lv, k, G):
    return np.ascontiguousarray(synth.pack2(lv[:, k * G:(k + 1) * G], G // 4))


def test_streaming_equals_one_shot(P):
    import torch

    nchan, G, ngulps = 64, 4096, 5
    f = synth.band_freqs(nchan)
    dms = synth.dm_list_linear(32, 60.0)
    plan = P.Plan(f, 64e-6, dms)
    lv = stream_levels(1, nchan, ngulps, G)
    total = ngulps * G - plan.maxdelay
    tap = torch.full((32, P.out_stride(total)), -1, dtype=torch.int32, device="cuda")
    srv = P.Server([plan], G, max_slots=2, half_window=512, max_cands=256)
    srv.set_tap(0, tap, total)
    seen = []
    for k in range(ngulps):
        while srv.submit(0, gulp_bytes(lv, k, G)) is None:
            seen += srv.poll(wait_s=0.5)
    srv.drain()
    seen += srv.poll()
    torch.cuda.synchronize()
    assert sorted(r["seq"] for r, _ in seen) == list(range(ngulps))
    for r, _ in seen:
        assert r["t0"] == (0 if r["seq"] == 0 else r["seq"] * G - plan.maxdelay)
        assert r["nout"] == (G - plan.maxdelay if r["seq"] == 0 else G)
    want = oracle.dedisperse(oracle.delay_table(f, 64e-6, dms), synth.pack2(lv), ngulps * G)
    np.testing.assert_array_equal(P.as_uint32(tap)[:, :total], want)
    srv.close()


def _run_server(P, plans, beam_gulps, order, ckpt):
    srv = P.Server(plans, 4096, max_slots=4, half_window=512, max_cands=512, classifier_path=ckpt)
    results = {}
    for beam, k in order:
        while srv.submit(beam, beam_gulps[beam][k]) is None:
            for r, c in srv.poll(wait_s=0.2):
                results[(r["beam"], r["seq"])] = c
    srv.drain()
    for r, c in srv.poll(max_results=256):
        results[(r["beam"], r["seq"])] = c
    srv.close()
    return results


def test_results_same_alone_and_in_the_mix(P, tmp_path):
    nchan, G, ngulps = 64, 4096, 4
    f = synth.band_freqs(nchan)
    plans = [P.Plan(f, 64e-6, synth.dm_list_linear(32 + 8 * b, 40.0 + 10 * b)) for b in range(5)]
    clf = P.Classifier(max_batch=64, seed=5)
    ckpt = str(tmp_path / "clf.ckpt")
    clf.save(ckpt)
    gulps = []
    for b in range(5):
        lv = stream_levels(10 + b, nchan, ngulps, G)
        gulps.append([gulp_bytes(lv, k, G) for k in range(ngulps)])
    alone = _run_server(P, plans[:1], gulps[:1], [(0, k) for k in range(ngulps)], ckpt)
    mix_order = [(b, k) for k in range(ngulps) for b in (3, 0, 4, 1, 2)]
    mixed = _run_server(P, plans, gulps, mix_order, ckpt)
    assert len(mixed) == 5 * ngulps
    for k in range(ngulps):
        a, m = alone[(0, k)], mixed[(0, k)]
        assert len(a) == len(m)
        for fld in ("d", "t", "w", "snr", "ncells", "score"):
            np.testing.assert_array_equal(a[fld], m[fld])
    assert any(len(alone[(0, k)]) for k in range(ngulps))


def test_admission_busy_when_slots_full(P):
    nchan, G = 64, 4096
    f = synth.band_freqs(nchan)
    plans = [P.Plan(f, 64e-6, synth.dm_list_linear(16, 30.0)) for _ in range(6)]
    srv = P.Server(plans, G, max_slots=1, half_window=256, max_cands=64)
    g = gulp_bytes(stream_levels(3, nchan, 1, G, with_pulses=False), 0, G)
    seqs = [srv.submit(b, g) for b in range(6)]
    assert seqs[0] == 0 and any(s is None for s in seqs[1:])
    srv.drain()
    srv.poll(max_results=16)
    assert srv.submit(5, g) is not None
    srv.drain()
    assert srv.info()["slots"] == 1
    srv.close()


def test_admission_respects_free_memory_and_rejects_bad_gulps(P):
    nchan, G = 64, 4096
    f = synth.band_freqs(nchan)
    plan = P.Plan(f, 64e-6, synth.dm_list_linear(16, 30.0))
    srv = P.Server([plan], G, max_slots=4, hbm_reserve=1 << 50, half_window=256)
    g = gulp_bytes(stream_levels(4, nchan, 1, G, with_pulses=False), 0, G)
    assert srv.submit(0, g) is None  # no slot fits under a 1 PiB reserve
    with pytest.raises(P.DDError):
        srv.submit(3, g)  # no such beam
    with pytest.raises(P.DDError):
        srv.submit(0, np.zeros((nchan, 8), np.uint8))  # rows shorter than a gulp
    srv.close()
    with pytest.raises(P.DDError):
        P.Server([plan], 100)  # gulp not a multiple of 64 / not above maxdelay


def test_triggered_dumps_hold_the_raw_sweep(P):
    """A bright dispersed pulse fires the trigger: each dump is the raw 2-bit
    input of the stream at absolute samples [t0, t0 + nsamp) (zeros before
    the stream starts) and contains the pulse's whole sweep; a threshold above
    every candidate fires nothing."""
    nchan, G, ngulps = 64, 4096, 4
    f = synth.band_freqs(nchan)
    dms = synth.dm_list_linear(32, 60.0)
    plan = P.Plan(f, 64e-6, dms)
    rng = np.random.default_rng(21)
    lv = synth.noise_levels(rng, nchan, ngulps * G)
    offs = oracle.delay_table(f, 64e-6, [40.0])[0]
    t_pulse = 9000
    synth.apply_recipe(lv, synth.BeamRecipe(pulses=[synth.Pulse(t0=t_pulse, offsets=offs, amp=2, width=8, dm=40.0)]))
    for thr, expect in ((20.0, True), (1e9, False)):
        dumps = []
        srv = P.Server([plan], G, max_slots=2, half_window=512, max_cands=256, trigger_snr=thr, trigger_max=3,
                       on_trigger=lambda info, raw: dumps.append((info, raw)))
        for k in range(ngulps):
            while srv.submit(0, gulp_bytes(lv, k, G)) is None:
                srv.poll(wait_s=0.5)
        srv.drain()
        srv.poll(max_results=16)
        srv.close()
        assert bool(dumps) == expect
        for info, raw in dumps:
            assert info["snr"] >= thr and raw.shape == (nchan, info["nsamp"] // 4)
            t0, ns = info["t0"], info["nsamp"]
            want_lv = np.zeros((nchan, ns), np.uint8)
            lo = max(t0, 0)
            want_lv[:, lo - t0:] = lv[:, lo:t0 + ns]
            np.testing.assert_array_equal(raw, synth.pack2(want_lv, ns // 4))
        if expect:
            info = max(dumps, key=lambda x: x[0]["snr"])[0]
            sweep = t_pulse + offs
            assert info["t0"] <= sweep.min() and sweep.max() + 8 <= info["t0"] + info["nsamp"]


def test_triggered_dumps_back_to_back(P):
    """Triggers fire in every gulp, on pulses placed so each dump starts
    inside the window's carried history, with up to four gulps of the beam in
    flight: every dump still equals the raw stream (the next gulp's history
    copy into that window waits for the dump)."""
    nchan, G, ngulps = 64, 4096, 10
    f = synth.band_freqs(nchan)
    dms = synth.dm_list_linear(32, 60.0)
    plan = P.Plan(f, 64e-6, dms)
    rng = np.random.default_rng(33)
    lv = synth.noise_levels(rng, nchan, ngulps * G)
    offs = oracle.delay_table(f, 64e-6, [30.0])[0]
    pulses = [synth.Pulse(t0=k * G - plan.maxdelay + 96, offsets=offs, amp=2, width=8, dm=30.0)
              for k in range(1, ngulps)]
    synth.apply_recipe(lv, synth.BeamRecipe(pulses=pulses))
    dumps = []
    srv = P.Server([plan], G, max_slots=4, half_window=512, max_cands=256, trigger_snr=15.0, trigger_max=2,
                   on_trigger=lambda info, raw: dumps.append((info, raw)))
    gulps = [gulp_bytes(lv, k, G) for k in range(ngulps)]
    for k in range(ngulps):
        while srv.submit(0, gulps[k]) is None:
            srv.poll(wait_s=0.05)
    srv.drain()
    srv.poll(max_results=64)
    srv.close()
    fired = sorted({info["seq"] for info, _ in dumps})
    assert fired == list(range(1, ngulps)), fired
    starts_in_history = 0
    for info, raw in dumps:
        t0, ns = info["t0"], info["nsamp"]
        want_lv = np.zeros((nchan, ns), np.uint8)
        lo = max(t0, 0)
        want_lv[:, lo - t0:] = lv[:, lo:t0 + ns]
        np.testing.assert_array_equal(raw, synth.pack2(want_lv, ns // 4))
        starts_in_history += int(t0 < info["seq"] * G)
    assert starts_in_history >= ngulps - 1


def test_streaming_1024_channels_candidates_equal_oracle(P):
    """The single-beam band (1024 channels, 700 trials to DM 249.5) streamed in
    four 2^15-sample gulps carrying the multibeam injection recipe (pulses,
    stuck channels, zero-DM bursts): the dedispersed stream equals the
    oracle's one-shot sums, and every gulp's complete candidate list equals
    the oracle's search of that gulp's output slice (baseline window clipped
    to the slice)."""
    import torch

    nchan, G, ngulps, half = 1024, 1 << 15, 4, 4096
    f = synth.band_freqs(nchan)
    dms = synth.dm_list_piecewise(250.0)
    plan = P.Plan(f, 64e-6, dms)
    rng = np.random.default_rng(77)
    total_in = ngulps * G
    lv = synth.noise_levels(rng, nchan, total_in)
    rec = synth.draw_recipe(rng, nchan, total_in - plan.maxdelay, 250.0,
                            lambda dm: oracle.delay_table(f, 64e-6, [dm])[0], npulses=12)
    synth.apply_recipe(lv, rec)
    total = total_in - plan.maxdelay
    tap = torch.full((len(dms), P.out_stride(total)), -1, dtype=torch.int32, device="cuda")
    srv = P.Server([plan], G, max_slots=3, half_window=half, max_cands=16384)
    srv.set_tap(0, tap, total)
    seen = []
    for k in range(ngulps):
        while srv.submit(0, gulp_bytes(lv, k, G)) is None:
            seen += srv.poll(wait_s=0.5)
    srv.drain()
    seen += srv.poll(max_results=16)
    srv.close()
    torch.cuda.synchronize()
    assert sorted(r["seq"] for r, _ in seen) == list(range(ngulps))
    x = oracle.dedisperse(oracle.delay_table(f, 64e-6, dms), synth.pack2(lv), total_in)
    np.testing.assert_array_equal(P.as_uint32(tap)[:, :total], x)
    widths = [1 << k for k in range(11)]
    ncand = 0
    for r, c in seen:
        assert r["flags"] == 0
        sl = np.ascontiguousarray(x[:, r["t0"]:r["t0"] + r["nout"]])
        y = oracle.baseline(sl, half)
        best, bw = oracle.best_snr(y, widths)
        want = oracle.find_peaks(best, bw, 6.0)
        assert len(c) == len(want) == r["ngroups"], (r["seq"], len(c), len(want))
        for fld in ("d", "t", "w", "snr", "ncells"):
            np.testing.assert_array_equal(c[fld], want[fld], err_msg=f"gulp {r['seq']} field {fld}")
        ncand += len(c)
    assert ncand > 0
