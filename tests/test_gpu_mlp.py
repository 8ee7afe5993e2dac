"""The warm-start MLP kernels (through the C ABI) against the numpy oracle
with the same bfloat16 rounding points: forward outputs, parameter gradients
and the Adam update.  Accumulation order differs (float32 sums), which can
flip a bfloat16 rounding of an activation; the bars allow for that and still
catch a transposed or dropped term (an O(1) error)."""
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
    out = tl.mlp_forward(_bf16_bits(theta), torch.as_tensor(x, device="cuda")).cpu().numpy()
    ref, _ = omlp.forward(theta, x, bf16=True)
    err = np.abs(out - ref)
    assert err.max() <= 2e-2 * np.abs(ref).max()
    assert err.mean() <= 2e-3 * np.abs(ref).mean()


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
    assert abs(loss.item() - ref_loss) <= 1e-2 * ref_loss
    assert np.linalg.norm(g - g_ref) <= 2e-2 * np.linalg.norm(g_ref)
    # per-layer blocks (a mistake in one layer shows up as an O(1) block error)
    bounds = np.cumsum([0] + [int(np.prod(s)) for s in omlp.SIZES])
    for a, b in zip(bounds[:-1], bounds[1:]):
        assert np.linalg.norm(g[a:b] - g_ref[a:b]) <= 5e-2 * np.linalg.norm(g_ref[a:b]) + 1e-7


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
