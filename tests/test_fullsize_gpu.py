"""Parity at full size, against the oracle:

* the whole single-beam output (1024 channels x 1500 DM trials x 2^19
  samples, the multibeam injection recipe applied) equals the oracle's sums;
* every beam of the 13-beam batched launch (graph replay) equals the oracle on
  32 whole DM rows spread over its range, first and last included;
* a 1024 x 1500 x 2^17 gulp with pulses, stuck channels and zero-DM bursts:
  the baseline-removed rows, their sums of squares and the complete candidate
  list (d, t, w, snr, ncells of every group) from the production search equal
  the oracle's, and so do the snippets of 300 random candidates and the 20
  brightest.

The search's input is the library's dedispersed output, which the first test
pins to the oracle bit for bit on the same shape.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

WIDTHS = tuple(1 << k for k in range(11))
HALF = 4096


@pytest.fixture(scope="module")
def P():
    import paper_1112_0065_gb300 as P

    P.load_library()
    return P


def _oracle_rows(delays, rows, packed, nout):
    """Oracle sums of the given DM rows over outputs [0, nout)."""
    sub = np.ascontiguousarray(delays[rows])
    return oracle.dedisperse(sub, packed, nout + int(sub.max()))


def _injected_gulp(P, f, plan, nout, seed, npulses=20):
    rng = np.random.default_rng(seed)
    nsamp = nout + plan.maxdelay
    d_in = synth.device_noise_packed(f.size, nsamp, seed=seed)
    rec = synth.draw_recipe(rng, f.size, nout, float(plan.dms[-1]) + 1.0,
                            lambda dm: oracle.delay_table(f, 64e-6, [dm])[0], npulses=npulses)
    synth.device_apply_recipe(d_in, nsamp, rec)
    return d_in, nsamp


def test_single_beam_whole_output_equals_oracle(P):
    import torch

    f = synth.band_freqs(1024)
    dms = synth.dm_list_piecewise(1000.0)
    plan = P.Plan(f, 64e-6, dms)
    d_in, nsamp = _injected_gulp(P, f, plan, 1 << 19, synth.BASE_SEED + 101)
    plan.autotune(nsamp)
    out = plan.execute(d_in, nsamp)
    torch.cuda.synchronize()
    packed = d_in.cpu().numpy()
    delays = oracle.delay_table(f, 64e-6, dms)
    nout = plan.nout(nsamp)
    assert nout == 1 << 19 and out.shape[0] == 1500
    for d0 in range(0, 1500, 125):
        rows = np.arange(d0, d0 + 125)
        want = _oracle_rows(delays, rows, packed, nout)
        got = P.as_uint32(out[d0:d0 + 125, :nout])
        if not np.array_equal(got, want):
            bad = np.argwhere(got != want)
            raise AssertionError(f"{len(bad)} outputs differ in rows {d0}..{d0 + 124}; first (row, t) "
                                 f"{tuple(bad[0] + [d0, 0])}")
    assert int(P.as_uint32(out[:, :nout]).max()) == 3 * 1024   # the zero-DM bursts saturate every channel
    plan.close()


def test_multibeam_every_beam_rows_equal_oracle(P):
    import torch

    from test_batch_gpu import multibeam_config

    f, cfg = multibeam_config()
    plans, items = {}, []
    rng = np.random.default_rng(11)
    for b, nout, dm_max, seed in cfg:
        if dm_max not in plans:
            plans[dm_max] = P.Plan(f, 64e-6, synth.dm_list_piecewise(dm_max))
        plan = plans[dm_max]
        nsamp = nout + plan.maxdelay
        d_in = synth.device_noise_packed(1024, nsamp, seed=seed)
        rec = synth.draw_recipe(rng, 1024, nout, dm_max, lambda dm: oracle.delay_table(f, 64e-6, [dm])[0])
        synth.device_apply_recipe(d_in, nsamp, rec)
        out = plan.alloc_output(nsamp)
        out.fill_(-1)
        items.append((plan, d_in, nsamp, out))
    batch = P.Batch(items, use_graph=True)
    batch.launch()
    batch.launch()   # a second replay over the same buffers
    torch.cuda.synchronize()
    assert len(items) == 13
    for plan, d_in, nsamp, out in items:
        delays = oracle.delay_table(f, 64e-6, plan.dms)
        n = plan.nout(nsamp)
        rows = np.unique(np.linspace(0, plan.ndm - 1, 32).round().astype(np.int64))
        want = _oracle_rows(delays, rows, d_in.cpu().numpy(), n)
        got = P.as_uint32(out[torch.as_tensor(rows, device="cuda"), :n])
        np.testing.assert_array_equal(got, want)
    batch.close()


def test_fullsize_candidates_equal_oracle(P):
    import torch

    f = synth.band_freqs(1024)
    dms = synth.dm_list_piecewise(1000.0)
    plan = P.Plan(f, 64e-6, dms)
    n = 1 << 17
    d_in, nsamp = _injected_gulp(P, f, plan, n, synth.BASE_SEED + 202, npulses=40)
    out = plan.execute(d_in, nsamp)
    s = P.Search(1500, n, nchan=1024, half_window=HALF, widths=WIDTHS, thresh=6.0, max_cands=1 << 17,
                 full_map=False)
    s.run(out, 1500, n)
    res = s.result()
    c = s.candidates()
    y, ss, _, _ = s.buffers()
    torch.cuda.synchronize()
    assert res["flags"] == 0
    x = P.as_uint32(out[:, :n])

    y_or = oracle.baseline(x, HALF)
    np.testing.assert_array_equal(y.cpu().numpy(), y_or)
    ss_or = (y_or.astype(np.int64) ** 2).sum(axis=1)
    np.testing.assert_array_equal(ss.cpu().numpy(), ss_or)
    best_or, bw_or = oracle.best_snr(y_or, WIDTHS)
    c_or = oracle.find_peaks(best_or, bw_or, 6.0)
    hot_or = int((best_or >= 6.0).sum())
    del best_or, bw_or

    assert res["nhot"] == hot_or
    assert res["ngroups"] == len(c_or) == len(c) and len(c) >= 256
    for k in ("d", "t", "w", "snr", "ncells"):
        np.testing.assert_array_equal(c[k], c_or[k], err_msg=k)

    rng = np.random.default_rng(3)
    pick = np.unique(np.concatenate([rng.choice(len(c), min(300, len(c)), replace=False),
                                     np.argsort(c["snr"])[-20:]]))
    sn = s.snippets(len(c))
    torch.cuda.synchronize()
    got = sn[torch.as_tensor(pick, device="cuda")].view(torch.int16).cpu().numpy().view(np.uint16)
    sn_or = oracle.snippets(y_or, ss_or, c_or["d"][pick], c_or["t"][pick], c_or["w"][pick])
    assert len(pick) >= 256
    np.testing.assert_array_equal(got, sn_or)
    s.close()
    plan.close()
