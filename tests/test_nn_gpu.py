"""The GPU classifier against the CPU oracle: forward logits bit-exact (same
bfloat16 rounding points and summation order), gradients within float
round-off of the oracle's, AdamW steps bit-exact, checkpoints round-trip, and
training on a separable toy set drives the loss down."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_1112_0065_gb300 as P

    P.load_library()
    return P


def params_with_biases(P, seed):
    p = P.init_params(seed)
    rng = np.random.default_rng(seed + 1000)
    off = 0
    for name, shp in P.classifier.SHAPES:
        k = int(np.prod(shp))
        if name.endswith(".b"):
            p[off:off + k] = rng.standard_normal(k).astype(np.float32) * 0.1
        off += k
    return p


def snippets(seed, n):
    rng = np.random.default_rng(seed)
    return oracle.float_to_bf16_bits(rng.standard_normal((n, 64, 64)).astype(np.float32) * 1.5)


def to_dev(bits):
    import torch

    return torch.from_numpy(bits.view(np.int16)).cuda().view(torch.bfloat16)


@pytest.mark.parametrize("n", [1, 37])
def test_forward_bit_exact(P, n):
    """The fixed-order forward (the one training uses) equals the oracle bit
    for bit."""
    import torch

    p = params_with_biases(P, 3)
    x = snippets(4, n)
    c = P.Classifier(max_batch=64, params=p)
    z = c.forward(to_dev(x))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(z.cpu().numpy(), oracle.nn_forward(p, x, round_bf16=True))


@pytest.mark.parametrize("scale,neg", [(100.0, False), (1.0, True)])
def test_forward_bit_exact_pooling_edges(P, scale, neg):
    """Inference pools the float maximum and rounds once; training rounds all
    four values and keeps the first maximum.  Both must give the oracle's
    logits: with 100x brighter inputs (many ties after rounding to bfloat16)
    and with weights flipped negative (most windows all <= 0, pooled to +0).
    The backward pass here runs the training forward on the same inputs."""
    import torch

    p = params_with_biases(P, 7)
    if neg:
        p = -np.abs(p)
    x = oracle.float_to_bf16_bits(oracle.bf16_bits_to_float(snippets(8, 40)) * scale)
    c = P.Classifier(max_batch=64, params=p)
    z = c.forward(to_dev(x))
    torch.cuda.synchronize()
    want = oracle.nn_forward(p, x, round_bf16=True)
    np.testing.assert_array_equal(z.cpu().numpy(), want)
    y = (np.arange(40) % 2).astype(np.float32)
    c.backward(to_dev(x), torch.from_numpy(y).cuda())
    loss_or, _, _ = oracle.nn_backward(p, x, y, round_bf16=True)
    assert abs(c.loss() - loss_or) <= 1e-6 * max(1.0, abs(loss_or))


def test_forward_bit_exact_at_launch_size(P):
    """One launch of the bench's size (8192 snippets: every persistent block
    walks many snippet groups, the last group ragged by a few snippets) and
    a second of 4099: 64 sampled logits of each equal the oracle's."""
    import torch

    p = params_with_biases(P, 5)
    c = P.Classifier(max_batch=8192, params=p)
    for n, seed in ((8192, 21), (4099, 22)):
        x = snippets(seed, n)
        z = c.forward(to_dev(x)).cpu().numpy()
        torch.cuda.synchronize()
        idx = np.unique(np.concatenate([np.random.default_rng(seed).choice(n, 60, replace=False),
                                        [0, 1, n - 2, n - 1]]))
        np.testing.assert_array_equal(z[idx], oracle.nn_forward(p, x[idx], round_bf16=True))


@pytest.mark.parametrize("n,seed", [(1, 11), (37, 12), (301, 13)])
def test_tensor_core_forward_drift_outside_logit_tolerance(P, n, seed):
    """NOT a parity test: the opt-in tensor-core forward does NOT meet the
    classifier's 1e-3 absolute logit tolerance and no served path uses it
    (servers and the benchmark's step score with the fixed-order forward,
    which is bit-exact against the oracle).  Its sums run in the tensor
    cores' order, so a float round-off difference now and then moves a
    bfloat16-rounded activation by one unit.  This test only bounds the drift
    it actually shows on these inputs: at most 5e-2 on any logit and at least
    60 % of logits within 1e-3 (on pipeline candidates with bright S/N maps
    the largest difference reaches about 0.6).  Odd batches leave a
    half-empty last tile in the deepest layer."""
    import torch

    p = params_with_biases(P, seed)
    x = snippets(seed + 50, n)
    c = P.Classifier(max_batch=512, params=p)
    z = c.forward(to_dev(x), tensor_cores=True)
    torch.cuda.synchronize()
    assert c.status() == 0
    want = oracle.nn_forward(p, x, round_bf16=True)
    err = np.abs(z.cpu().numpy() - want)
    assert float(err.max()) <= 5e-2, float(err.max())
    assert float(np.mean(err <= 1e-3)) >= 0.6, float(np.mean(err <= 1e-3))


def test_tensor_core_forward_drift_scales_with_the_logits(P):
    """NOT a parity test (see above): with inputs 100x larger (bright S/N
    maps) the tensor-core logits stay within 3 % of the logit scale of the
    oracle's, which is far outside 1e-3 absolute."""
    import torch

    p = params_with_biases(P, 21)
    x = oracle.float_to_bf16_bits(oracle.bf16_bits_to_float(snippets(22, 64)) * 100.0)
    c = P.Classifier(max_batch=64, params=p)
    z = c.forward(to_dev(x), tensor_cores=True).cpu().numpy()
    assert c.status() == 0
    want = oracle.nn_forward(p, x, round_bf16=True)
    scale = float(np.abs(want).max())
    assert float(np.abs(z - want).max()) <= 3e-2 * scale, (float(np.abs(z - want).max()), scale)


def test_backward_matches_oracle(P):
    import torch

    p = params_with_biases(P, 5)
    x = snippets(6, 24)
    y = (np.arange(24) % 3 == 0).astype(np.float32)
    c = P.Classifier(max_batch=64, params=p)
    c.backward(to_dev(x), torch.from_numpy(y).cuda())
    g = c.grads()
    loss = c.loss()
    loss_or, g_or, _ = oracle.nn_backward(p, x, y, round_bf16=True)
    assert abs(loss - loss_or) <= 1e-6 * max(1.0, abs(loss_or))
    off = 0
    for name, shp in P.classifier.SHAPES:
        k = int(np.prod(shp))
        a, b = g[off:off + k], g_or[off:off + k]
        scale = float(np.max(np.abs(b))) + 1e-12
        assert float(np.max(np.abs(a - b))) <= 1e-4 * scale, name
        off += k


def test_adamw_bit_exact(P):
    rng = np.random.default_rng(8)
    p = params_with_biases(P, 9)
    c = P.Classifier(max_batch=8, params=p)
    master = p.copy()
    m = np.zeros_like(master)
    v = np.zeros_like(master)
    for step in (1, 2, 3):
        g = (rng.standard_normal(master.size) * 1e-2).astype(np.float32)
        c.set_grads(g)
        c.adamw(1e-3, 0.9, 0.999, 1e-8, 0.01)
        bits = oracle.adamw_step(master, g, m, v, 1e-3, 0.9, 0.999, 1e-8, 0.01, step)
        gm, gv, gb, st = c.state()
        assert st == step
        np.testing.assert_array_equal(c.params(), master)
        np.testing.assert_array_equal(gm, m)
        np.testing.assert_array_equal(gv, v)
        np.testing.assert_array_equal(gb, bits)


def test_checkpoint_round_trip(P, tmp_path):
    import torch

    c = P.Classifier(max_batch=8, params=params_with_biases(P, 11))
    c.set_grads(np.full(P.classifier.NN_PARAMS, 1e-3, np.float32))
    c.adamw(1e-3)
    path = str(tmp_path / "clf.ckpt")
    c.save(path)
    d = P.Classifier(max_batch=8)
    d.load(path)
    np.testing.assert_array_equal(d.params(), c.params())
    assert d.state()[3] == 1
    x = to_dev(snippets(12, 5))
    np.testing.assert_array_equal(d.forward(x).cpu().numpy(), c.forward(x).cpu().numpy())
    with pytest.raises(P.DDError):
        d.load(str(tmp_path / "missing.ckpt"))
    del torch


def toy_batch(rng, n):
    """Positives: a bright compact blob at the centre with a bow-tie of
    fainter DM sidelobes; negatives: noise, or a bright band along time (a
    zero-DM burst seen across DM rows)."""
    x = rng.standard_normal((n, 64, 64)).astype(np.float32)
    y = (rng.random(n) < 0.5).astype(np.float32)
    for i in range(n):
        if y[i]:
            for r in range(64):
                spread = 1 + abs(r - 32) // 4
                x[i, r, 32 - spread:32 + spread] += 6.0 / spread
        elif rng.random() < 0.5:
            t = rng.integers(5, 59)
            x[i, :, t - 2:t + 2] += 3.0
    return oracle.float_to_bf16_bits(x), y


def test_training_reduces_loss(P):
    import torch

    rng = np.random.default_rng(13)
    c = P.Classifier(max_batch=128, seed=1)
    losses = []
    for step in range(40):
        xb, yb = toy_batch(rng, 64)
        c.train_step(to_dev(xb), torch.from_numpy(yb).cuda(), lr=2e-3)
        losses.append(c.loss())
    assert np.mean(losses[-5:]) < 0.5 * np.mean(losses[:5])
    xt, yt = toy_batch(np.random.default_rng(99), 128)
    z = c.forward(to_dev(xt)).cpu().numpy()
    assert np.mean((z > 0) == (yt > 0.5)) > 0.9
