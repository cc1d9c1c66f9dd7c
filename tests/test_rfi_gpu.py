"""The GPU coincidence RFI mask against the oracle: zero-DM series, the mask
and its count, and the in-place substitution, bit-exact -- on designed bursts
over 13 beams of 1024 channels, on noise with a loose threshold (many
coincidences), and on ragged lengths."""
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


def make_beams(seed, nbeams, nchan, nsamp, events):
    rng = np.random.default_rng(seed)
    out = []
    for b in range(nbeams):
        lv = synth.noise_levels(rng, nchan, nsamp)
        for t0, dur, bs in events:
            if b in bs:
                lv[:, t0:t0 + dur] = 3
        out.append(synth.pack2(lv))
    return out


def check(P, beams, nsamp, k, m):
    import torch

    nchan = beams[0].shape[0]
    dev = [torch.from_numpy(b).cuda() for b in beams]
    r = P.RfiMask(16, nchan, nsamp + 100)
    r.run(dev, nsamp, k_sigma=k, min_beams=m, apply=True)
    nm = r.nmasked()
    z, mask = r.buffers()
    torch.cuda.synchronize()
    z_or = np.stack([oracle.zero_dm(b, nsamp) for b in beams])
    mask_or, nm_or = oracle.rfi_mask(z_or, k, m)
    np.testing.assert_array_equal(z.cpu().numpy().view(np.uint32), z_or)
    np.testing.assert_array_equal(mask.cpu().numpy(), mask_or)
    assert nm == nm_or
    for b, d in zip(beams, dev):
        np.testing.assert_array_equal(d.cpu().numpy(), oracle.rfi_apply(b, nsamp, mask_or))
    r.close()
    return nm


def test_bursts_over_13_beams(P):
    nsamp = 20000
    events = [(1000, 40, set(range(5))), (2500, 30, {0, 4, 8, 12}), (9000, 50, {1, 2, 3}), (15000, 20, {7}),
              (19990, 10, set(range(13)))]
    nm = check(P, make_beams(7, 13, 1024, nsamp, events), nsamp, 3, 4)
    assert nm == 80


@pytest.mark.parametrize("nsamp,nchan,k,m", [(40001, 64, 1, 4), (17, 7, 1, 1), (4096, 130, 0, 13)])
def test_loose_thresholds_and_ragged_sizes(P, nsamp, nchan, k, m):
    check(P, make_beams(nsamp + nchan, 13, nchan, nsamp, [(0, 3, {0, 1, 2, 3})]), nsamp, k, m)
