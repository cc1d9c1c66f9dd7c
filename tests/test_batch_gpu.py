"""Batched persistent multi-beam dedispersion: each beam's result equals the
oracle (small beams, in full) and equals the single-gulp path bit-exactly (the
13-beam multibeam configuration), with and without CUDA-graph replay, and after
the batch's buffers are swapped."""
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


SMALL = [  # seed, nchan, ndm, dm_end, nsamp
    (1, 64, 40, 100.0, 8192),
    (2, 64, 17, 30.0, 3001),
    (3, 64, 64, 60.0, 5555),
    (4, 64, 9, 0.0, 777),
    (5, 64, 33, 90.0, 12000),
]


def _small_beams(P, shape=(16, 2), chan_chunk=64):
    import torch

    f = synth.band_freqs(64)
    beams, wants = [], []
    for seed, nchan, ndm, dm_end, nsamp in SMALL:
        dms = synth.dm_list_linear(ndm, dm_end)
        plan = P.Plan(f, 64e-6, dms, kernel=P.KERNEL_TILED, dms_per_block=shape[0], words_per_thread=shape[1],
                      chan_chunk=chan_chunk)
        packed, _ = synth.make_gulp(seed, nchan, nsamp)
        d_in = torch.from_numpy(packed).cuda()
        out = plan.alloc_output(nsamp)
        out.fill_(-1)
        beams.append((plan, d_in, nsamp, out))
        wants.append(oracle.dedisperse(oracle.delay_table(f, 64e-6, dms), packed, nsamp))
    return beams, wants


def _check(P, beams, wants):
    import torch

    torch.cuda.synchronize()
    for (plan, _, nsamp, out), want in zip(beams, wants):
        np.testing.assert_array_equal(P.as_uint32(out)[:, : plan.nout(nsamp)], want)


@pytest.mark.parametrize("use_graph", [False, True])
def test_small_batch_matches_oracle(P, use_graph):
    beams, wants = _small_beams(P, shape=(16, 2) if use_graph else (8, 3))
    b = P.Batch(beams, use_graph=use_graph)
    info = b.info()
    assert info["nbeams"] == len(SMALL) and info["grid"] >= 152
    b.launch()
    _check(P, beams, wants)
    for _, _, _, out in beams:
        out.fill_(-1)
    b.launch()  # replay
    _check(P, beams, wants)
    b.close()


@pytest.mark.parametrize("chan_chunk", [32, 128])
def test_small_batch_other_channel_chunks(P, chan_chunk):
    beams, wants = _small_beams(P, shape=(16, 3), chan_chunk=chan_chunk)
    b = P.Batch(beams, use_graph=True)
    b.launch()
    _check(P, beams, wants)
    b.close()


def test_batch_of_different_bands(P):
    """Beams with different channel counts, bands, sampling times and DM
    grids in one persistent launch: every beam's shared-memory layout (slot,
    channel bases) differs while the stage mbarriers, at the start of shared
    memory, carry their phases from one beam's tiles to the next."""
    import torch

    beams, wants = [], []
    for seed, nchan, ndm, dm_end, nsamp, tsamp in [(21, 64, 40, 100.0, 8192, 64e-6), (22, 130, 23, 60.0, 5000, 64e-6),
                                                   (23, 200, 70, 150.0, 12345, 128e-6), (24, 7, 5, 40.0, 1001, 64e-6)]:
        f = synth.band_freqs(nchan)
        dms = synth.dm_list_linear(ndm, dm_end)
        plan = P.Plan(f, tsamp, dms, kernel=P.KERNEL_TILED, dms_per_block=8, words_per_thread=5, chan_chunk=64)
        packed, _ = synth.make_gulp(seed, nchan, nsamp)
        out = plan.alloc_output(nsamp)
        out.fill_(-1)
        beams.append((plan, torch.from_numpy(packed).cuda(), nsamp, out))
        wants.append(oracle.dedisperse(oracle.delay_table(f, tsamp, dms), packed, nsamp))
    b = P.Batch(beams, use_graph=True)
    b.launch()
    _check(P, beams, wants)
    for _, _, _, out in beams:
        out.fill_(-1)
    b.launch()
    _check(P, beams, wants)
    assert P.dedisp_status() == 0
    b.close()


def test_autotune_after_batch_keeps_its_tables(P):
    """Tuning a plan while a batch built on it is alive keeps the tables the
    batch's descriptors point at: the batch still gives the oracle's sums."""
    import torch

    f = synth.band_freqs(64)
    dms = synth.dm_list_linear(40, 100.0)
    plan = P.Plan(f, 64e-6, dms)   # default shape, tables built at creation
    nsamp = 8192
    packed, _ = synth.make_gulp(41, 64, nsamp)
    d_in = torch.from_numpy(packed).cuda()
    out = plan.alloc_output(nsamp)
    b = P.Batch([(plan, d_in, nsamp, out)], use_graph=True)
    plan.autotune(nsamp)
    junk = [torch.zeros(1 << 20, dtype=torch.int32, device="cuda") for _ in range(8)]  # reuse of freed memory
    out.fill_(-1)
    b.launch()
    _check(P, [(plan, d_in, nsamp, out)], [oracle.dedisperse(oracle.delay_table(f, 64e-6, dms), packed, nsamp)])
    b.close()
    del junk


def test_batch_set_swaps_buffers(P):
    import torch

    beams, wants = _small_beams(P)
    b = P.Batch(beams, use_graph=True)
    b.launch()
    # new inputs for the same plans, fewer beams, fresh outputs
    new_beams, new_wants = [], []
    f = synth.band_freqs(64)
    for (plan, _, nsamp, _), (seed, nchan, ndm, dm_end, _) in list(zip(beams, SMALL))[:3]:
        packed, _ = synth.make_gulp(seed + 100, nchan, nsamp)
        out = plan.alloc_output(nsamp)
        new_beams.append((plan, torch.from_numpy(packed).cuda(), nsamp, out))
        new_wants.append(oracle.dedisperse(oracle.delay_table(f, 64e-6, synth.dm_list_linear(ndm, dm_end)),
                                           packed, nsamp))
    b.set(new_beams)
    b.launch()
    _check(P, new_beams, new_wants)
    b.close()


def test_execute_batch_one_shot(P):
    beams, wants = _small_beams(P, shape=(8, 2))
    P.execute_batch(beams)
    _check(P, beams, wants)


def test_batch_rejects_mixed_shapes_and_bad_beams(P):
    import torch

    beams, _ = _small_beams(P)
    plan, d_in, nsamp, out = beams[0]
    with pytest.raises(P.DDError):
        P.Batch([(plan, d_in, plan.maxdelay, out)])  # too short
    simple = P.Plan(synth.band_freqs(64), 64e-6, [0.0, 1.0], kernel=P.KERNEL_SIMPLE)
    with pytest.raises(P.DDError):
        P.Batch([(simple, d_in, nsamp, out)])
    del torch


def multibeam_config(seed_base=synth.BASE_SEED + 3000):
    """13 beams over the 1024-channel band; per beam: output length uniform
    in [2^16, 2^19], maximum DM drawn from {250, 500, 1000} with the
    0.25/0.5/1.0 step rule, independent noise, 20 dispersed pulses, 5% stuck
    channels and 3 zero-DM bursts."""
    rng = np.random.default_rng(seed_base)
    f = synth.band_freqs(1024)
    beams = []
    for b in range(13):
        nout = int(rng.integers(1 << 16, (1 << 19) + 1))
        dm_max = float(rng.choice([250.0, 500.0, 1000.0]))
        beams.append((b, nout, dm_max, int(seed_base + b)))
    return f, beams


def test_multibeam_batch_equals_single_gulp(P):
    import torch

    f, cfg = multibeam_config()
    plans = {}
    items, solos = [], []
    rng = np.random.default_rng(7)
    for b, nout, dm_max, seed in cfg:
        if dm_max not in plans:
            plans[dm_max] = P.Plan(f, 64e-6, synth.dm_list_piecewise(dm_max))
        plan = plans[dm_max]
        nsamp = nout + plan.maxdelay
        d_in = synth.device_noise_packed(1024, nsamp, seed=seed)
        rec = synth.draw_recipe(rng, 1024, nout, dm_max,
                                lambda dm: oracle.delay_table(f, 64e-6, [dm])[0])
        synth.device_apply_recipe(d_in, nsamp, rec)
        out = plan.alloc_output(nsamp)
        items.append((plan, d_in, nsamp, out))
    batch = P.Batch(items, use_graph=True)
    batch.launch()
    torch.cuda.synchronize()
    for plan, d_in, nsamp, out in items:
        solo = plan.execute(d_in, nsamp)
        torch.cuda.synchronize()
        n = plan.nout(nsamp)
        assert torch.equal(solo[:, :n], out[:, :n])
        del solo
    # and a sample of every beam against the oracle
    for plan, d_in, nsamp, out in items[:4]:
        packed = d_in.cpu().numpy()
        delays = oracle.delay_table(f, 64e-6, plan.dms)
        n = plan.nout(nsamp)
        di = rng.integers(0, plan.ndm, 300)
        ti = rng.integers(0, n, 300)
        want = oracle.dedisperse_points(delays, packed, nsamp, di, ti)
        got = out[torch.as_tensor(di, device="cuda").long(), torch.as_tensor(ti, device="cuda").long()]
        np.testing.assert_array_equal(got.cpu().numpy().view(np.uint32), want)
    batch.close()
