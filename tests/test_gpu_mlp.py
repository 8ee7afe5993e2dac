"""The warm-start MLP kernels (through the C ABI) against the numpy oracle
with the same bfloat16 rounding points: forward outputs, the stored bfloat16
activations, parameter gradients and the Adam update; then the start's input,
target and extrapolation kernels against the oracle.  The float32 sums run in
another order, which can move a sum across a bfloat16 rounding boundary: the
bars count such activation flips (at most one bfloat16 unit each, in at most
0.1 % of the activations) and bound the outputs and gradients a few hundred
times below what one dropped or transposed term would cause."""
import numpy as np
import pytest

from oracle import mlp as omlp

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _tl():
    from paper_2604_10357_gb300 import build, tl
    build.build()
    return tl


def _bf16_bits(theta):
    r = omlp.bf16_round(theta.astype(np.float32))
    return torch.as_tensor((r.view(np.uint32) >> 16).astype(np.uint16).view(np.int16), device="cuda")


@pytest.fixture(scope="module")
def setup():
    rng = np.random.default_rng(50)
    theta = omlp.init_params(rng)
    theta += (0.05 * rng.normal(size=theta.shape)).astype(np.float32)
    n = 1000   # several blocks of 128 and a ragged tail
    x = rng.normal(size=(n, 10)).astype(np.float32)
    x[:, 9] = rng.integers(0, 2, size=n)
    target = rng.normal(size=(n, 3)).astype(np.float32)
    w = np.full(n, 1.0 / n, np.float32)
    return theta, x, target, w


def test_forward_matches_oracle(setup):
    tl = _tl()
    theta, x, _, _ = setup
    acts = torch.empty(x.shape[0], 192, dtype=torch.int16, device="cuda")
    out = tl.mlp_forward(_bf16_bits(theta), torch.as_tensor(x, device="cuda"), acts=acts).cpu().numpy()
    ref, cache = omlp.forward(theta, x, bf16=True)
    err = np.abs(out - ref)
    assert err.max() <= 1e-5 * np.abs(ref).max()
    # the stored activations are the oracle's bfloat16 values, up to rare one-unit flips
    a = (acts.cpu().numpy().view(np.uint16).astype(np.uint32) << 16).view(np.float32)
    refa = np.concatenate([cache[1], cache[2], cache[3]], axis=1)
    diff = np.abs(a - refa)
    assert np.count_nonzero(diff) <= 1e-3 * diff.size
    assert np.all(diff <= 2.0 ** -7 * np.maximum(np.abs(refa), 2.0 ** -126))


def test_backward_matches_oracle(setup):
    tl = _tl()
    theta, x, target, w = setup
    P = _bf16_bits(theta)
    xd = torch.as_tensor(x, device="cuda")
    acts = torch.empty(x.shape[0], 192, dtype=torch.int16, device="cuda")
    out = tl.mlp_forward(P, xd, acts=acts)
    dout = torch.empty_like(out)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    tl.mlp_mse_grad(out, torch.as_tensor(target, device="cuda"), torch.as_tensor(w, device="cuda"), dout, loss)
    grads = torch.zeros(omlp.NPARAM, dtype=torch.float32, device="cuda")
    tl.mlp_backward(P, xd, acts, dout, grads)
    torch.cuda.synchronize()
    ref_out, cache = omlp.forward(theta, x, bf16=True)
    ref_loss, ref_dout = omlp.mse(ref_out, target, w)
    g_ref = omlp.backward(theta, cache, ref_dout)
    g = grads.cpu().numpy()
    assert abs(loss.item() - ref_loss) <= 1e-6 * ref_loss
    assert np.linalg.norm(g - g_ref) <= 1e-5 * np.linalg.norm(g_ref)
    # per-layer blocks (a mistake in one layer shows up as an O(1) block error)
    bounds = np.cumsum([0] + [int(np.prod(s)) for s in omlp.SIZES])
    for a, b in zip(bounds[:-1], bounds[1:]):
        assert np.linalg.norm(g[a:b] - g_ref[a:b]) <= 1e-4 * np.linalg.norm(g_ref[a:b]) + 1e-9


def test_adam_matches_oracle():
    tl = _tl()
    rng = np.random.default_rng(51)
    n = omlp.NPARAM
    master = rng.normal(size=n).astype(np.float32)
    g = rng.normal(size=n).astype(np.float32)
    m1 = 0.01 * rng.normal(size=n).astype(np.float32)
    m2 = np.abs(0.01 * rng.normal(size=n)).astype(np.float32)
    dev = [torch.as_tensor(a.copy(), device="cuda") for a in (master, g, m1, m2)]
    P = torch.empty(n, dtype=torch.int16, device="cuda")
    tl.mlp_adam(dev[0], P, dev[1], dev[2], dev[3], lr=1e-3, step=3)
    ref = omlp.adam_step(master.copy(), g, m1.copy(), m2.copy(), 3, lr=1e-3)
    assert np.allclose(dev[0].cpu().numpy(), ref, rtol=1e-5, atol=1e-6)
    bits = P.cpu().numpy().view(np.uint16).astype(np.uint32) << 16
    assert np.array_equal(bits.view(np.float32), omlp.bf16_round(dev[0].cpu().numpy()))


@pytest.fixture(scope="module")
def history_case():
    """A 525-node box with its x = 0 face clamped and a random velocity history."""
    tl = _tl()
    from paper_2604_10357_gb300 import inputs
    m = inputs.box_t10(10, 2, 2, 1.0, 0.1, 0.1)
    g = tl.Mesh(m.X, m.conn, [dict(inputs.SVK_1E7)], precision=tl.TL_FP64)
    g.build_pattern(m.fixed_nodes)
    rng = np.random.default_rng(52)
    hist = [rng.normal(scale=s, size=(m.nn, 3)) for s in (1.0, 0.9, 1.1, 0.8)]
    for h in hist:
        h[m.fixed_nodes] = 0.0
    v_next = rng.normal(size=(m.nn, 3))
    fixed = np.zeros(m.nn, bool)
    fixed[m.fixed_nodes] = True
    return tl, g, hist, v_next, fixed


def _d(a):
    return None if a is None else torch.as_tensor(np.ascontiguousarray(a).reshape(-1), device="cuda")


@pytest.mark.parametrize("order", [1, 2, 3, 4])
def test_features_and_target_match_oracle(history_case, order):
    """tl_mlp_features and tl_mlp_target against the oracle with 1..4 history
    velocities (the missing ones NULL): both round the same float64 values to
    float32, so they agree to one float32 rounding."""
    tl, g, hist, v_next, fixed = history_case
    h = hist[:order] + [None] * (4 - order)
    sc = (0.7, 1.3, 2.9)
    f = g.mlp_features([_d(a) for a in h], sc).cpu().numpy()
    ref = omlp.features(*h, fixed, *sc)
    assert np.all(np.abs(f - ref) <= 2.0 ** -22 * np.abs(ref) + 1e-300)
    t = g.mlp_target(_d(v_next), [_d(a) for a in h], sc, 0.37).cpu().numpy()
    tref = omlp.target(v_next, *h, fixed, *sc, 0.37)
    assert np.all(np.abs(t - tref) <= 2.0 ** -22 * np.abs(tref) + 1e-300)
    assert np.all(t[fixed] == 0.0) and np.all(f[fixed, 9] == 1.0) and np.all(f[~fixed, 9] == 0.0)


@pytest.mark.parametrize("order", [1, 2, 3, 4])
def test_warm_start_extrapolation_matches_oracle(history_case, order):
    """tl_warm_start without a network: the polynomial extrapolation of the
    available history, 0 on clamped nodes (float64, same arithmetic)."""
    tl, g, hist, _, fixed = history_case
    h = hist[:order] + [None] * (4 - order)
    v0 = g.warm_start(None, [_d(a) for a in h]).cpu().numpy().reshape(-1, 3)
    ref = omlp.start_velocity(None, *h, fixed, 1.0, 1.0, 1.0, 1.0)
    assert np.abs(v0 - ref).max() <= 1e-14 * np.abs(ref).max()
    assert np.all(v0[fixed] == 0.0)


def test_warm_start_with_network_matches_oracle(history_case):
    """tl_warm_start with a network: extrapolation + s_out * MLP(features), the
    forward pass emulated by the oracle with the same bfloat16 rounding."""
    tl, g, hist, _, fixed = history_case
    rng = np.random.default_rng(53)
    theta = omlp.init_params(rng) + (0.05 * rng.normal(size=omlp.NPARAM)).astype(np.float32)
    sc, s_out = (0.7, 1.3, 2.9), 0.05
    v0 = g.warm_start(_bf16_bits(theta), [_d(a) for a in hist], sc, s_out).cpu().numpy().reshape(-1, 3)
    feats = omlp.features(*hist, fixed, *sc).astype(np.float32)
    out, _ = omlp.forward(theta, feats, bf16=True)
    ref = omlp.start_velocity(out, *hist, fixed, *sc, s_out)
    corr = s_out * np.abs(out * omlp.node_scale(*hist, *sc)[:, None]).max()
    assert np.all(v0[fixed] == 0.0)
    assert np.abs(v0 - ref).max() <= 2e-2 * corr


def test_col_sumsq():
    tl = _tl()
    rng = np.random.default_rng(54)
    x = rng.normal(size=(3001, 7)).astype(np.float32)
    out = torch.zeros(7, dtype=torch.float64, device="cuda")
    tl.mlp_col_sumsq(torch.as_tensor(x, device="cuda"), out)
    tl.mlp_col_sumsq(torch.as_tensor(x, device="cuda"), out)      # accumulates
    ref = 2.0 * np.sum(x.astype(np.float64) ** 2, axis=0)
    assert np.allclose(out.cpu().numpy(), ref, rtol=1e-12)
