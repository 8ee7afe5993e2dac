"""Pins of the warm-start MLP oracle: float64 gradients against central
finite differences, the bfloat16 rounding routine against its definition, and
the start's inputs and base: backward differences against their closed forms
on cubic histories, the extrapolation's exactness on polynomial histories, the
feature layout on a history built by hand, and the start / target round trip."""
import numpy as np
import pytest

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


def _poly_history(rng, deg, n=5):
    """Velocities v_k = P(k) at k = 0, -1, -2, -3 for a random polynomial of
    degree deg per node and component; returns the history, P(1) and the
    coefficients (a, b, c, d) of a + b t + c t^2 + d t^3."""
    coef = [rng.normal(size=(n, 3)) if k <= deg else np.zeros((n, 3)) for k in range(4)]
    P = lambda t: coef[0] + coef[1] * t + coef[2] * t ** 2 + coef[3] * t ** 3   # noqa: E731
    return [P(0.0), P(-1.0), P(-2.0), P(-3.0)], P(1.0), coef


def test_backward_differences_of_a_cubic():
    """For P(t) = a + b t + c t^2 + d t^3 sampled at t = 0, -1, -2, -3:
    nabla P = b - c + d, nabla^2 P = 2c - 6d, nabla^3 P = 6d."""
    rng = np.random.default_rng(41)
    hist, _, (a, b, c, d) = _poly_history(rng, 3)
    d1, d2, d3 = mlp.backward_differences(*hist)
    assert np.allclose(d1, b - c + d, rtol=0, atol=1e-12)
    assert np.allclose(d2, 2 * c - 6 * d, rtol=0, atol=1e-12)
    assert np.allclose(d3, 6 * d, rtol=0, atol=1e-12)


@pytest.mark.parametrize("deg", [0, 1, 2, 3])
def test_extrapolation_is_exact_for_polynomial_histories(deg):
    """With the deg + 1 most recent velocities of a polynomial history of
    degree deg, the extrapolation reproduces P(1) (Newton's backward-difference
    formula); with all four it is exact for every degree <= 3."""
    rng = np.random.default_rng(42 + deg)
    hist, nxt, _ = _poly_history(rng, deg)
    partial = hist[:deg + 1] + [None] * (3 - deg)
    assert np.allclose(mlp.extrapolation(*partial), nxt, rtol=0, atol=1e-11)
    assert np.allclose(mlp.extrapolation(*hist), nxt, rtol=0, atol=1e-11)
    if deg >= 1:   # one velocity fewer than the degree needs: not exact
        short = hist[:deg] + [None] * (4 - deg)
        assert np.abs(mlp.extrapolation(*short) - nxt).max() > 1e-3


def test_features_layout_on_a_hand_built_history():
    """Two nodes, velocities chosen by hand: node 0's velocity has the constant
    second difference (2, 0, -1) from v_{n-3} = (1, 1, 1) on; node 1 is fixed
    and at rest.  Columns: nabla v / s1, nabla^2 v / s2, nabla^3 v / s3, flag."""
    v3 = np.array([[1.0, 1.0, 1.0], [0.0, 0.0, 0.0]])
    v2 = np.array([[3.0, 1.0, 0.0], [0.0, 0.0, 0.0]])
    v1 = np.array([[7.0, 1.0, -2.0], [0.0, 0.0, 0.0]])
    v0 = np.array([[13.0, 1.0, -5.0], [0.0, 0.0, 0.0]])
    f = mlp.features(v0, v1, v2, v3, np.array([False, True]), 2.0, 0.5, 4.0)
    # scaled differences (3, 0, -1.5 | 4, 0, -2 | 0, 0, 0), norm sqrt(9 + 2.25 + 16 + 4) = 5.59...
    r = np.sqrt(31.25)
    expect = np.array([[3.0 / r, 0.0, -1.5 / r, 4.0 / r, 0.0, -2.0 / r, 0.0, 0.0, 0.0, 0.0],
                       [0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0]])
    assert np.allclose(f, expect, rtol=0, atol=1e-15)
    assert np.allclose(mlp.node_scale(v0, v1, v2, v3, 2.0, 0.5, 4.0), [r, 0.0], rtol=0, atol=1e-14)
    # missing history: the differences that need it are zero (norm 3.354...)
    f2 = mlp.features(v0, v1, None, None, np.array([False, True]), 2.0, 0.5, 4.0)
    assert np.array_equal(f2[:, 3:9], np.zeros((2, 6)))
    assert np.allclose(f2[0, :3], np.array([3.0, 0.0, -1.5]) / np.sqrt(11.25), rtol=0, atol=1e-15)
    # the inputs do not depend on the amplitude of the motion
    assert np.allclose(mlp.features(7 * v0, 7 * v1, 7 * v2, 7 * v3, np.array([False, True]), 2.0, 0.5, 4.0), f,
                       rtol=0, atol=1e-15)


def test_start_velocity_round_trip_and_fixed_nodes():
    """The start built from the exact target reproduces v_{n+1} on free nodes;
    fixed nodes start at rest whatever the network says."""
    rng = np.random.default_rng(43)
    hist = [rng.normal(size=(6, 3)) for _ in range(4)]
    v_next = rng.normal(size=(6, 3))
    fixed = np.array([True, False, False, True, False, False])
    sc = (0.5, 2.0, 3.0)
    t = mlp.target(v_next, *hist, fixed, *sc, 0.25)
    v0 = mlp.start_velocity(t, *hist, fixed, *sc, 0.25)
    assert np.allclose(v0[~fixed], v_next[~fixed], rtol=0, atol=1e-12)
    assert np.array_equal(v0[fixed], np.zeros((2, 3))) and np.array_equal(t[fixed], np.zeros((2, 3)))
    assert np.array_equal(mlp.start_velocity(rng.normal(size=(6, 3)), *hist, fixed, *sc, 3.0)[fixed],
                          np.zeros((2, 3)))
    # the same motion 10x larger: the same target (the correction scales with the history)
    t10 = mlp.target(10 * v_next, *(10 * h for h in hist), fixed, *sc, 0.25)
    assert np.allclose(t10, t, rtol=1e-12, atol=1e-15)
