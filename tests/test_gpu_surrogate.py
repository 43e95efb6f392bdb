"""The surrogate network's BF16 tensor-core kernels against the FP64 oracle
network (GPU, through the C ABI).

Parameters and inputs are rounded to BF16 first, so both sides start from the
same values; the GPU then rounds activations and activation gradients to BF16
at every layer (8 bits of mantissa), so outputs must agree to a relative L2
error of 3e-2 and parameter gradients to 6e-2 per tensor (cosine >= 0.995).

Every element is bounded too.  BF16's unit roundoff is u = 2^-8; an output
passes through about nine such roundings (two per convolution of each level
and the head), so an element's error is about 3 u = 0.012 of its tensor's RMS
and the largest of some 10^4 elements about 4.5 times that, 0.05: outputs
must stay within 0.10 of their tensor's RMS at every element.  Parameter
gradients also carry the rounded activation gradients and the forward error
entering the loss gradient (y - target), whose relative error grows where y
and the target nearly cancel.  A weight-gradient element of the deepest
level sums few products (32 pixels at 16 x 16 inputs, batch 2), so single
elements there deviate by up to about 1.2 of the tensor's RMS while the
tensor as a whole stays within its L2 bound; every element must stay within
1.5 of the RMS.  (A worst-case running error bound, propagated through |W|
at every layer, exceeds the gradients themselves by orders of magnitude at
this depth and cannot serve.)"""
import numpy as np
import pytest

from oracle import surrogate as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

WIDTHS = (32, 64, 128)


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def bf16_round(a):
    t = torch.as_tensor(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float32)
    return t.numpy().astype(np.float64)


def flatten(P, widths, cin, cout):
    parts = []
    for name, ci, co in S.layer_names(widths):
        parts += [P[name + ".W"].reshape(-1), P[name + ".b"]]
    parts += [P["head.W"].reshape(-1), P["head.b"]]
    return np.concatenate(parts)


def unflatten(vec, widths, cin, cout):
    G, o = {}, 0
    for name, ci, co in S.layer_names(widths):
        ci = cin if ci is None else ci
        n = 9 * ci * co
        G[name + ".W"] = vec[o:o + n].reshape(3, 3, ci, co)
        o += n
        G[name + ".b"] = vec[o:o + co]
        o += co
    G["head.W"] = vec[o:o + widths[0] * cout].reshape(widths[0], cout)
    o += widths[0] * cout
    G["head.b"] = vec[o:o + cout]
    return G


def make(seed=0, size=16, batch=2, widths=WIDTHS):
    import paper_2301_08343_gb300 as T
    net = T.SurrogateNet(widths, 2, 3, size=size, max_batch=4, seed=seed)
    P = S.init_params(widths, 2, 3, seed=seed)
    rng = np.random.default_rng(seed + 1)
    for k in P:
        if k.endswith(".b"):
            P[k] = rng.normal(0, 0.05, P[k].shape)
        P[k] = bf16_round(P[k])
    net.set_params(flatten(P, widths, 2, 3))
    x = bf16_round(rng.normal(size=(batch, size, size, 2)))
    t = rng.normal(size=(batch, size, size, 3)) * 0.5
    return net, P, x, t


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def elementwise(a, b):
    """Largest element error of a against b, in units of b's RMS."""
    a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
    return float(np.abs(a - b).max() / max(np.sqrt(np.mean(b * b)), 1e-30))


def check_gradients(G, Go):
    for k in Go:
        a, b = G[k].ravel(), Go[k].ravel()
        cos = float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-30))
        assert rel(a, b) <= 6e-2, (k, rel(a, b))
        assert cos >= 0.995, (k, cos)
        assert elementwise(a, b) <= 1.5, (k, elementwise(a, b))


def test_parameter_count_and_layout():
    import paper_2301_08343_gb300 as T
    net = T.SurrogateNet((32, 64, 128, 256), 2, 3, size=64, max_batch=2)
    P = S.init_params((32, 64, 128, 256), 2, 3, seed=0)
    assert net.num_params == sum(v.size for v in P.values())
    assert 1.8e6 < net.num_params < 2.1e6


def test_forward_matches_oracle():
    net, P, x, t = make()
    y = net.forward(x).cpu().numpy()
    yo, _ = S.forward(P, x, WIDTHS)
    assert rel(y, yo) <= 3e-2
    assert elementwise(y, yo) <= 0.10, elementwise(y, yo)


def test_gradients_match_oracle():
    net, P, x, t = make(seed=3)
    loss = net.gradients(x, t)
    lo, Go = S.loss_and_grad(P, x, t, WIDTHS)
    assert abs(loss - lo) <= 3e-2 * lo
    G = unflatten(net.get_params(grads=True).astype(np.float64), WIDTHS, 2, 3)
    check_gradients(G, Go)


def test_four_levels_match_oracle():
    # the full widths: output-channel tiles of 32 ... 256 and, in the data
    # gradient of the bottom decoder layer (384 input channels), two tiles of 192
    # (32 x 32 images: the bottom level keeps 4 x 4 pixels, so its weight
    # gradients are sums over enough terms for the BF16 noise to average)
    widths = (32, 64, 128, 256)
    net, P, x, t = make(seed=7, size=32, widths=widths)
    y = net.forward(x).cpu().numpy()
    yo, _ = S.forward(P, x, widths)
    assert rel(y, yo) <= 3e-2
    assert elementwise(y, yo) <= 0.10, elementwise(y, yo)
    net.gradients(x, t)
    _, Go = S.loss_and_grad(P, x, t, widths)
    G = unflatten(net.get_params(grads=True).astype(np.float64), widths, 2, 3)
    check_gradients(G, Go)


def test_full_size_matches_oracle():
    # the configuration the benchmark trains: 64 x 64 maps, widths up to 256
    # (levels 64, 32, 16 and 8 pixels wide: the pixel boxes of the 3x3
    # convolution kernels are 2, 4, 8 and 16 image rows)
    widths = (32, 64, 128, 256)
    net, P, x, t = make(seed=11, size=64, batch=2, widths=widths)
    y = net.forward(x).cpu().numpy()
    yo, _ = S.forward(P, x, widths)
    assert rel(y, yo) <= 3e-2
    assert elementwise(y, yo) <= 0.10, elementwise(y, yo)
    net.gradients(x, t)
    _, Go = S.loss_and_grad(P, x, t, widths)
    G = unflatten(net.get_params(grads=True).astype(np.float64), widths, 2, 3)
    check_gradients(G, Go)


def test_adam_steps_reduce_the_loss_and_match_the_oracle_step():
    net, P, x, t = make(seed=5)
    l0 = net.train_step(x, t, lr=1e-3)
    p1 = net.get_params().astype(np.float64)
    # the oracle's first Adam step from the same gradients moves every
    # parameter by lr * sign(g) (within eps); compare signs and magnitudes
    _, Go = S.loss_and_grad(P, x, t, WIDTHS)
    p0 = flatten(P, WIDTHS, 2, 3)
    g0 = flatten(Go, WIDTHS, 2, 3)
    step = p1 - p0
    big = np.abs(g0) > 1e-3 * np.abs(g0).max()
    assert np.mean(np.sign(step[big]) == -np.sign(g0[big])) >= 0.99
    assert np.allclose(np.abs(step[big]), 1e-3, rtol=2e-2)
    losses = [l0] + [net.train_step(x, t, lr=1e-3) for _ in range(30)]
    assert losses[-1] < 0.5 * losses[0]


def test_full_size_forward_is_finite_and_batch_consistent():
    import paper_2301_08343_gb300 as T
    net = T.SurrogateNet((32, 64, 128, 256), 2, 3, size=64, max_batch=8, seed=1)
    x = torch.randn(8, 64, 64, 2, device="cuda")
    y = net.forward(x)
    y1 = net.forward(x[3:4])
    assert torch.isfinite(y).all()
    assert torch.allclose(y[3:4], y1, rtol=0, atol=1e-5)
