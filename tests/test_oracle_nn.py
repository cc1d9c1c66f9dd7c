"""Pins for the classifier oracle (CPU only): the unrounded forward pass
against scipy's 2-D correlation + numpy pooling/matmul in float64, the
backward pass against central finite differences, closed forms for zero
weights, the loss and one AdamW step, and bfloat16 rounding against an
independent bit-level statement."""
import numpy as np
import pytest

import oracle

signal = pytest.importorskip("scipy.signal")


def he_init(seed):
    rng = np.random.default_rng(seed)
    parts = []
    for name, shp in oracle.NN_SHAPES:
        if name.endswith(".w"):
            fan_in = int(np.prod(shp[1:]))
            parts.append(rng.standard_normal(int(np.prod(shp))) * np.sqrt(2.0 / fan_in))
        else:
            parts.append(rng.standard_normal(int(np.prod(shp))) * 0.05)
    return np.concatenate(parts).astype(np.float32)


def rand_x(seed, n):
    rng = np.random.default_rng(seed)
    return oracle.float_to_bf16_bits(rng.standard_normal((n, 64, 64)).astype(np.float32))


def numpy_forward(params, xbits):
    P = {k: v.astype(np.float64) for k, v in oracle.nn_split(params).items()}
    x = oracle.bf16_bits_to_float(xbits).astype(np.float64)
    out = []
    for n in range(x.shape[0]):
        a = x[n][None]
        for l in range(1, 5):
            w, b = P[f"conv{l}.w"], P[f"conv{l}.b"]
            co = np.stack([sum(signal.correlate2d(a[ci], w[o, ci], mode="same") for ci in range(a.shape[0])) + b[o]
                           for o in range(w.shape[0])])
            co = np.maximum(co, 0)
            H = co.shape[1]
            a = co.reshape(co.shape[0], H // 2, 2, H // 2, 2).max(axis=(2, 4))
        feat = a.reshape(-1)
        h = np.maximum(P["fc1.w"] @ feat + P["fc1.b"], 0)
        out.append(float(P["fc2.w"][0] @ h + P["fc2.b"][0]))
    return np.array(out)


def test_param_count():
    assert oracle.nn_param_count() == 191553 == sum(int(np.prod(s)) for _, s in oracle.NN_SHAPES)


def test_forward_matches_scipy_unrounded():
    p = he_init(1)
    x = rand_x(2, 3)
    got = oracle.nn_forward(p, x, round_bf16=False)
    want = numpy_forward(p, x)
    np.testing.assert_allclose(got, want, rtol=1e-4, atol=1e-4)


def test_forward_rounded_close_to_unrounded():
    p = he_init(3)
    x = rand_x(4, 4)
    a = oracle.nn_forward(p, x, round_bf16=True)
    b = numpy_forward(p, x)
    assert np.max(np.abs(a - b)) < 0.05 * (1 + np.max(np.abs(b)))


def test_zero_weights_give_the_output_bias():
    p = np.zeros(oracle.nn_param_count(), dtype=np.float32)
    p[-1] = 0.37
    z = oracle.nn_forward(p, rand_x(5, 2), round_bf16=True)
    assert np.all(z == oracle.bf16_bits_to_float(oracle.float_to_bf16_bits(np.float32(0.37))))
    assert abs(oracle.nn_loss(np.zeros(4, np.float32), np.array([0, 1, 0, 1], np.float32)) - np.log(2)) < 1e-6


def test_loss_closed_form():
    z = np.array([-3.0, -0.5, 0.0, 2.0, 7.0], dtype=np.float32)
    y = np.array([0, 1, 1, 0, 1], dtype=np.float32)
    want = np.mean(-(y * np.log(1 / (1 + np.exp(-z.astype(np.float64)))) +
                     (1 - y) * np.log(1 - 1 / (1 + np.exp(-z.astype(np.float64))))))
    assert abs(oracle.nn_loss(z, y) - want) < 1e-6


def test_backward_matches_finite_differences():
    p = he_init(7)
    x = rand_x(8, 2)
    y = np.array([1.0, 0.0], dtype=np.float32)
    loss, g, z = oracle.nn_backward(p, x, y, round_bf16=False)
    assert abs(loss - oracle.nn_loss(z, y)) < 1e-6
    rng = np.random.default_rng(0)
    checked = 0
    off = 0
    for name, shp in oracle.NN_SHAPES:
        k = int(np.prod(shp))
        gt = g[off:off + k]
        idx = list(np.argsort(-np.abs(gt))[:3]) + list(rng.integers(0, k, 2))
        for i in idx:
            j = off + int(i)
            eps = 1e-3 * max(1.0, abs(float(p[j])))
            pp, pm = p.copy(), p.copy()
            pp[j] += eps
            pm[j] -= eps
            lp = oracle.nn_loss(oracle.nn_forward(pp, x, False), y)
            lm = oracle.nn_loss(oracle.nn_forward(pm, x, False), y)
            fd = (lp - lm) / (2 * eps)
            # the network is piecewise linear: a step crosses some ReLU/max-pool kinks, so FD agrees to a few %
            atol = 1e-4 + 2e-3 * float(np.max(np.abs(gt)))  # float round-off of the loss difference
            assert abs(fd - g[j]) <= atol + 0.05 * abs(g[j]), (name, int(i), fd, g[j])
            checked += 1
        off += k
    assert checked == sum(min(3, int(np.prod(s))) + 2 for _, s in oracle.NN_SHAPES)


def test_adamw_first_step_closed_form():
    rng = np.random.default_rng(9)
    w = rng.standard_normal(1000).astype(np.float32)
    g = rng.standard_normal(1000).astype(np.float32)
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    w0 = w.copy()
    lr, wd, eps = 1e-3, 0.01, 1e-8
    bits = oracle.adamw_step(w, g, m, v, lr, 0.9, 0.999, eps, wd, 1)
    want = w0 - lr * (g / (np.abs(g) + eps) + wd * w0)
    np.testing.assert_allclose(w, want, rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-6)
    np.testing.assert_allclose(v, 0.001 * g * g, rtol=1e-4)  # 1 - 0.999 evaluated in float
    np.testing.assert_array_equal(bits, oracle.float_to_bf16_bits(w))


def test_bf16_rounding_ties_to_even():
    # 1 + 2^-8 lies halfway between 1 and 1 + 2^-7: ties go to the even mantissa (1.0)
    assert oracle.float_to_bf16_bits(np.float32(1 + 2 ** -8)) == 0x3F80
    # 1 + 3*2^-8 lies halfway between 1 + 2^-7 and 1 + 2^-6: even is 1 + 2^-6
    assert oracle.float_to_bf16_bits(np.float32(1 + 3 * 2 ** -8)) == 0x3F82
    assert oracle.float_to_bf16_bits(np.float32(-2.0)) == 0xC000
