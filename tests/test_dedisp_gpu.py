"""Bit-exact parity of the CUDA dedispersion path against the CPU oracle.

Inputs are seeded synthetic 2-bit gulps (synth); expected values come only from
the oracle.  Covers the tiny 64-channel configuration in full, ragged and
degenerate shapes for every tiled-kernel shape, and the 1024-channel x 1500-DM
x 2^19-sample single-beam configuration on sampled outputs and full rows.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TILED_SHAPES = [(8, 2), (16, 1), (16, 2), (32, 1), (8, 4), (8, 3), (16, 3), (8, 5)]  # (DMs per CTA, words per lane)
CHAN_CHUNKS = (64, 32, 128)  # channels per shared-memory stage
TILED_SHAPES_G = [(d, w, g) for g in CHAN_CHUNKS for (d, w) in TILED_SHAPES]


@pytest.fixture(scope="module")
def P():
    import paper_1112_0065_gb300 as P

    P.load_library()
    return P


def _run(P, plan, packed, nsamp):
    import torch

    d_in = torch.from_numpy(packed).cuda()
    out = plan.execute(d_in, nsamp)
    torch.cuda.synchronize()
    return P.as_uint32(out)[:, : plan.nout(nsamp)]


def tiny_config():
    nchan, nsamp = 64, 8192
    f = synth.band_freqs(nchan)
    dms = synth.dm_list_linear(64, 100.0)
    delays = oracle.delay_table(f, 64e-6, dms)
    rec = synth.BeamRecipe(pulses=[synth.Pulse(t0=1000, offsets=delays[32], amp=2, width=1, dm=50.0)])
    packed, _ = synth.make_gulp(synth.BASE_SEED, nchan, nsamp, rec)
    return f, dms, delays, packed, nsamp


def test_delay_table_matches_oracle(P):
    f = synth.band_freqs(1024)
    dms = synth.dm_list_piecewise(1000.0)
    plan = P.Plan(f, 64e-6, dms)
    np.testing.assert_array_equal(plan.delay_table(), oracle.delay_table(f, 64e-6, dms))
    assert plan.maxdelay == 20464


def test_delay_rounding_mode_golden(P):
    """The library's delay tables (plan upload and dd_compute_delays) hold the
    nearest integer of the exact delays in tests/golden/delay_rounding.txt."""
    from test_oracle_dedisp import _delay_rounding_golden, golden_delay_grid

    rows = _delay_rounding_golden()
    for key in sorted({(r[0], r[1]) for r in rows}):
        f, dms = golden_delay_grid(*key)
        plan = P.Plan(f, 64e-6, dms)
        tab = plan.delay_table()
        host = P.compute_delays(f, 64e-6, dms)
        plan.close()
        for nchan, grid, d, c, _, rounded, _, _ in rows:
            if (nchan, grid) == key:
                assert tab[d, c] == rounded and host[d, c] == rounded, (key, d, c)


@pytest.mark.parametrize("kernel", ["simple", "auto"] + [f"tiled{s}" for s in TILED_SHAPES_G])
def test_tiny_config_bit_exact(P, kernel):
    f, dms, delays, packed, nsamp = tiny_config()
    if kernel == "simple":
        plan = P.Plan(f, 64e-6, dms, kernel=P.KERNEL_SIMPLE)
    elif kernel == "auto":
        plan = P.Plan(f, 64e-6, dms)
    else:
        dpb, w, g = eval(kernel[5:])
        plan = P.Plan(f, 64e-6, dms, kernel=P.KERNEL_TILED, dms_per_block=dpb, words_per_thread=w, chan_chunk=g)
        assert plan.kernel_shape() == (P.KERNEL_TILED, dpb, w, g)
    want = oracle.dedisperse(delays, packed, nsamp)
    got = _run(P, plan, packed, nsamp)
    np.testing.assert_array_equal(got, want)
    assert got[32, 1000] == want.max()


def _case(seed, nchan, ndm, nsamp, dm_end, background="noise"):
    f = synth.band_freqs(nchan)
    dms = synth.dm_list_linear(ndm, dm_end)
    delays = oracle.delay_table(f, 64e-6, dms)
    packed, _ = synth.make_gulp(seed, nchan, nsamp, background=background)
    return f, dms, delays, packed


RAGGED = [
    # seed, nchan, ndm, nsamp, dm_end
    (1, 1, 1, 17, 0.0),         # single channel, single DM, maxdelay 0
    (2, 7, 3, 1001, 40.0),
    (3, 63, 17, 2049, 80.0),
    (4, 65, 33, 3333, 120.0),
    (5, 130, 9, 5000, 60.0),
    (6, 129, 40, 1537, 10.0),
    (7, 200, 70, 12345, 150.0),
]


@pytest.mark.parametrize("shape", [None] + TILED_SHAPES_G)
@pytest.mark.parametrize("case", RAGGED)
def test_ragged_shapes_bit_exact(P, case, shape):
    seed, nchan, ndm, nsamp, dm_end = case
    f, dms, delays, packed = _case(seed, nchan, ndm, nsamp, dm_end)
    if nsamp <= delays.max():
        pytest.skip("too short")
    if shape is None:
        plan = P.Plan(f, 64e-6, dms, kernel=P.KERNEL_SIMPLE)
    else:
        try:
            plan = P.Plan(f, 64e-6, dms, kernel=P.KERNEL_TILED, dms_per_block=shape[0], words_per_thread=shape[1],
                          chan_chunk=shape[2])
        except P.DDError as e:
            # two 128-channel stages of a wide delay spread exceed shared memory: refused, not run
            if shape[2] == 128 and "delay spread too large" in str(e):
                pytest.skip("128-channel stages do not fit shared memory for this spread")
            raise
    np.testing.assert_array_equal(_run(P, plan, packed, nsamp), oracle.dedisperse(delays, packed, nsamp))


@pytest.mark.parametrize("shape", [(16, 2, 64), (32, 1, 64), (16, 3, 64), (16, 3, 32), (8, 5, 32), (16, 3, 128),
                                   (32, 1, 128)])
def test_all_threes_saturates_exactly(P, shape):
    """Every sample at the top level: every output is 3*nchan (largest sums the
    bit-planes and the 16-bit lanes ever hold)."""
    nchan, ndm, nsamp = 1024, 24, 4000
    f = synth.band_freqs(nchan)
    dms = synth.dm_list_linear(ndm, 2.0)
    packed, _ = synth.make_gulp(0, nchan, nsamp, background="max")
    plan = P.Plan(f, 64e-6, dms, kernel=P.KERNEL_TILED, dms_per_block=shape[0], words_per_thread=shape[1],
                  chan_chunk=shape[2])
    got = _run(P, plan, packed, nsamp)
    assert np.all(got == 3 * nchan)


def test_large_nchan_and_irregular_dm_steps(P):
    rng = np.random.default_rng(9)
    nchan, nsamp = 1500, 9000
    f = synth.band_freqs(nchan)
    dms = np.sort(np.concatenate([[0.0, 0.0], rng.uniform(0, 150, 45)]))
    delays = oracle.delay_table(f, 64e-6, dms)
    packed, _ = synth.make_gulp(10, nchan, nsamp)
    plan = P.Plan(f, 64e-6, dms)
    np.testing.assert_array_equal(_run(P, plan, packed, nsamp), oracle.dedisperse(delays, packed, nsamp))


@pytest.mark.parametrize("shape", [(16, 2), (8, 2), (8, 5)])
def test_more_than_2047_channels(P, shape):
    """Bands wider than 2047 channels use the 15-plane variant."""
    nchan, ndm, nsamp = 2500, 20, 3000
    f = synth.band_freqs(nchan, bw=100.0)
    dms = synth.dm_list_linear(ndm, 30.0)
    delays = oracle.delay_table(f, 64e-6, dms)
    packed, _ = synth.make_gulp(21, nchan, nsamp)
    plan = P.Plan(f, 64e-6, dms, kernel=P.KERNEL_TILED, dms_per_block=shape[0], words_per_thread=shape[1])
    np.testing.assert_array_equal(_run(P, plan, packed, nsamp), oracle.dedisperse(delays, packed, nsamp))
    lv3, _ = synth.make_gulp(0, nchan, nsamp, background="max")
    assert np.all(_run(P, plan, lv3, nsamp) == 3 * nchan)


def test_wide_band_rejects_other_chunks(P):
    """Bands of 2048 channels or more run with 64-channel stages only."""
    f = synth.band_freqs(2500, bw=100.0)
    with pytest.raises(P.DDError):
        P.Plan(f, 64e-6, synth.dm_list_linear(8, 5.0), kernel=P.KERNEL_TILED, dms_per_block=16,
               words_per_thread=2, chan_chunk=32)
    with pytest.raises(P.DDError):
        P.Plan(synth.band_freqs(64), 64e-6, [0.0, 1.0], kernel=P.KERNEL_TILED, chan_chunk=48)


def test_autotuner_sweeps_channel_chunks(P):
    """The tuner times every (DMs, words, channel chunk) shape; its choice is
    one of them and gives the oracle's sums on a 1024-channel band."""
    f = synth.band_freqs(1024)
    dms = synth.dm_list_linear(96, 300.0)
    delays = oracle.delay_table(f, 64e-6, dms)
    nsamp = 40000
    packed, _ = synth.make_gulp(31, 1024, nsamp)
    plan = P.Plan(f, 64e-6, dms)
    ms = plan.autotune(nsamp)
    kern, dpb, w, g = plan.kernel_shape()
    assert ms > 0 and kern == P.KERNEL_AUTO and g in CHAN_CHUNKS and (dpb, w) in TILED_SHAPES
    np.testing.assert_array_equal(_run(P, plan, packed, nsamp), oracle.dedisperse(delays, packed, nsamp))


def test_wider_row_stride_and_offset_output(P):
    import torch

    f, dms, delays, packed = _case(12, 48, 20, 3000, 50.0)
    nsamp = 3000
    wide = np.zeros((48, packed.shape[1] + 64), dtype=np.uint8)
    wide[:, : packed.shape[1]] = packed
    plan = P.Plan(f, 64e-6, dms)
    d_in = torch.from_numpy(wide).cuda()
    nout = plan.nout(nsamp)
    big = torch.full((20, P.out_stride(nout) + 104), -1, dtype=torch.int32, device="cuda")
    out = big[:, 4:4 + P.out_stride(nout)]  # 16-byte aligned view with a wider row stride
    plan.execute(d_in, nsamp, out)
    torch.cuda.synchronize()
    got = P.as_uint32(big)
    np.testing.assert_array_equal(got[:, 4:4 + nout], oracle.dedisperse(delays, packed, nsamp))
    assert np.all(got[:, :4] == 0xFFFFFFFF) and np.all(got[:, 4 + nout:] == 0xFFFFFFFF)


def test_execute_host_matches_device(P):
    f, dms, delays, packed, nsamp = tiny_config()
    plan = P.Plan(f, 64e-6, dms)
    h = plan.execute_host(packed, nsamp)
    np.testing.assert_array_equal(h.numpy().view(np.uint32)[:, : plan.nout(nsamp)],
                                  oracle.dedisperse(delays, packed, nsamp))


def test_two_streams_same_plan(P):
    import torch

    f, dms, delays, packed, nsamp = tiny_config()
    plan = P.Plan(f, 64e-6, dms)
    d_in = torch.from_numpy(packed).cuda()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    o1 = plan.execute(d_in, nsamp, stream=s1)
    o2 = plan.execute(d_in, nsamp, stream=s2)
    torch.cuda.synchronize()
    want = oracle.dedisperse(delays, packed, nsamp)
    np.testing.assert_array_equal(P.as_uint32(o1)[:, : want.shape[1]], want)
    np.testing.assert_array_equal(P.as_uint32(o2)[:, : want.shape[1]], want)


def test_argument_errors(P):
    import torch

    f, dms, delays, packed, nsamp = tiny_config()
    plan = P.Plan(f, 64e-6, dms)
    d_in = torch.from_numpy(packed).cuda()
    out = plan.alloc_output(nsamp)
    with pytest.raises(P.DDError) as e:
        plan.execute(d_in, plan.maxdelay, out)
    assert e.value.status == -4
    with pytest.raises(P.DDError) as e:
        plan.execute(d_in, plan.maxdelay)   # empty output: NULL pointer
    assert e.value.status == -1
    with pytest.raises(P.DDError) as e:
        plan.execute(d_in[:, 4:], nsamp - 16, out)  # stride ok but misaligned base
    assert e.value.status == -1


def test_single_beam_htru_sampled(P):
    """1024 channels, 1500 DMs (piecewise 0.25/0.5/1.0), 2^19 output samples:
    ~3000 sampled outputs (including every corner) and three whole rows."""
    import torch

    nchan = 1024
    f = synth.band_freqs(nchan)
    dms = synth.dm_list_piecewise(1000.0)
    plan = P.Plan(f, 64e-6, dms)
    nsamp = (1 << 19) + plan.maxdelay
    d_in = synth.device_noise_packed(nchan, nsamp, seed=synth.BASE_SEED + 2)
    plan.autotune(nsamp)
    out = plan.execute(d_in, nsamp)
    torch.cuda.synchronize()
    packed = d_in.cpu().numpy()
    delays = oracle.delay_table(f, 64e-6, dms)
    nout = plan.nout(nsamp)
    assert nout == 1 << 19
    rng = np.random.default_rng(5)
    d_idx = np.concatenate([rng.integers(0, 1500, 3000), [0, 0, 1499, 1499, 750]])
    t_idx = np.concatenate([rng.integers(0, nout, 3000), [0, nout - 1, 0, nout - 1, nout // 2]])
    want = oracle.dedisperse_points(delays, packed, nsamp, d_idx, t_idx)
    got_all = out[torch.as_tensor(d_idx, device="cuda").long(), torch.as_tensor(t_idx, device="cuda").long()]
    np.testing.assert_array_equal(got_all.cpu().numpy().view(np.uint32), want)
    for row in (0, 777, 1499):
        t_full = np.arange(nout)
        want_row = oracle.dedisperse_points(delays, packed, nsamp, np.full(nout, row), t_full)
        np.testing.assert_array_equal(P.as_uint32(out[row, :nout]), want_row)


@pytest.mark.parametrize("nchan,nsamp", [(1024, 20000), (7, 33), (130, 4097)])
def test_corner_turn_then_dedisperse(P, nchan, nsamp):
    """Time-major input through the corner turn: the channel-major rows equal
    the oracle's, and dedispersing them equals the oracle's sums."""
    import torch

    rng = np.random.default_rng(nchan + nsamp)
    lv = rng.integers(0, 4, size=(nsamp, nchan)).astype(np.uint8)
    tm = synth.pack2(lv, (nchan + 3) // 4 + 5)
    cm = P.corner_turn(torch.from_numpy(tm).cuda(), nchan, nsamp)
    torch.cuda.synchronize()
    want = oracle.corner_turn(tm, nchan, nsamp, cm.shape[1])
    np.testing.assert_array_equal(cm.cpu().numpy(), want)
    f = synth.band_freqs(nchan)
    dms = synth.dm_list_linear(16, 20.0)
    plan = P.Plan(f, 64e-6, dms)
    if plan.maxdelay < nsamp:
        got = _run(P, plan, cm.cpu().numpy(), nsamp)
        np.testing.assert_array_equal(got, oracle.dedisperse(oracle.delay_table(f, 64e-6, dms), want, nsamp))


def test_autotune_cache_round_trip(P, tmp_path):
    """The tuner writes its choice to the plan's cache file; a new plan of the
    same band, DMs and gulp length reads it back (no timing, 0 ms) and runs
    the same shape, with the oracle's sums."""
    cache = str(tmp_path / "tune.txt")
    f = synth.band_freqs(256)
    dms = synth.dm_list_linear(48, 120.0)
    nsamp = 30000
    delays = oracle.delay_table(f, 64e-6, dms)
    packed, _ = synth.make_gulp(44, 256, nsamp)
    a = P.Plan(f, 64e-6, dms, tune_cache=cache)
    assert a.autotune(nsamp) > 0
    shape = a.kernel_shape()
    with open(cache) as fh:
        assert len(fh.read().strip().splitlines()) == 1
    b = P.Plan(f, 64e-6, dms, tune_cache=cache)
    assert b.autotune(nsamp) == 0.0
    assert b.kernel_shape() == shape
    np.testing.assert_array_equal(_run(P, b, packed, nsamp), oracle.dedisperse(delays, packed, nsamp))


def test_stage_waits_report_no_error(P):
    """The tiled kernels stage each channel window by a bulk copy whose
    completion every thread waits for with a bounded poll: after this
    module's launches (every tile shape, ragged sizes, batches of stages) the
    device error word is clear, and reading it clears it."""
    f, dms, delays, packed, nsamp = tiny_config()
    plan = P.Plan(f, 64e-6, dms)
    got = _run(P, plan, packed, nsamp)
    np.testing.assert_array_equal(got, oracle.dedisperse(delays, packed, nsamp))
    assert P.dedisp_status() == 0
    assert P.dedisp_status() == 0
    plan.close()


def test_tile_gives_up_without_fault(P):
    """The give-up path of the tile's bounded stage waits, run without any
    fault: the probe's tile waits on stage mbarriers that expect one arrival
    more than its copies make, so every wait runs out of polls; the tile sets
    bit 0 of its error word, writes no output, and the GPU context stays
    usable (the library's own error word is untouched and a dedispersion
    afterwards is still exact)."""
    from paper_1112_0065_gb300 import probes

    st, err, written, msg = probes.tile_giveup(1000)
    assert st == -5 and err == 1 and written == 0, (st, err, written, msg)
    assert "gave up" in msg
    assert P.dedisp_status() == 0
    f, dms, delays, packed, nsamp = tiny_config()
    plan = P.Plan(f, 64e-6, dms)
    np.testing.assert_array_equal(_run(P, plan, packed, nsamp), oracle.dedisperse(delays, packed, nsamp))
    plan.close()
