"""Pins of the warm-start MLP oracle: float64 gradients against central
finite differences, and the bfloat16 rounding routine against its definition."""
import numpy as np

from oracle import mlp


def test_backward_matches_central_differences():
    rng = np.random.default_rng(40)
    theta = mlp.init_params(rng).astype(np.float64)
    theta += 0.1 * rng.normal(size=theta.shape)
    x = rng.normal(size=(7, 10))
    target = rng.normal(size=(7, 3))
    w = rng.uniform(0.5, 1.0, size=7)

    def loss(t):
        out, _ = mlp.forward(t, x, bf16=False, dtype=np.float64)
        return mlp.mse(out, target, w)[0]

    out, cache = mlp.forward(theta, x, bf16=False, dtype=np.float64)
    _, dout = mlp.mse(out, target, w)
    g = mlp.backward(theta, cache, dout)
    idx = rng.choice(mlp.NPARAM, size=60, replace=False)
    idx = np.concatenate([idx, [0, 639, 640, 700, 4800, mlp.NPARAM - 4, mlp.NPARAM - 1]])
    eps = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += eps
        tm[i] -= eps
        fd = (loss(tp) - loss(tm)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_bf16_rounding_definition():
    # representable values are fixed points; halfway cases round to even
    vals = np.array([1.0, -2.5, 3.140625, 0.0], np.float32)
    assert np.array_equal(mlp.bf16_round(vals), vals)
    one = np.float32(1.0).view(np.uint32)
    half_up = np.array([one + 0x8000], np.uint32).view(np.float32)       # tie: 1 + 2^-8 -> 1 (even)
    assert mlp.bf16_round(half_up)[0] == 1.0
    odd = np.array([one + 0x10000 + 0x8000], np.uint32).view(np.float32)  # tie above odd -> up
    assert mlp.bf16_round(odd)[0] == np.array([one + 0x20000], np.uint32).view(np.float32)[0]
    just_above = np.array([one + 0x8001], np.uint32).view(np.float32)
    assert mlp.bf16_round(just_above)[0] == np.array([one + 0x10000], np.uint32).view(np.float32)[0]
    rng = np.random.default_rng(1)
    x = rng.normal(size=1000).astype(np.float32)
    r = mlp.bf16_round(x)
    assert np.all((r.view(np.uint32) & 0xFFFF) == 0)
    assert np.all(np.abs(r - x) <= np.abs(x) * 2.0 ** -8)


def test_adam_first_step_is_signed_lr():
    theta = np.zeros(5, np.float32)
    g = np.array([1.0, -2.0, 0.5, -0.1, 3.0], np.float32)
    m, v = np.zeros(5, np.float32), np.zeros(5, np.float32)
    mlp.adam_step(theta, g, m, v, 1, lr=0.01)
    assert np.allclose(theta, -0.01 * np.sign(g), rtol=1e-5)
