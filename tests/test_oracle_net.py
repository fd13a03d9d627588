"""Pin the FP64 proposal network: analytic gradients against finite
differences, the wrapped Cauchy density and its sampler."""
import numpy as np
import pytest

from oracle import net


def small_params(seed=0, scale=0.1):
    rng = np.random.default_rng(seed)
    return rng.normal(size=net.n_params()) * scale


def test_param_count_layout():
    assert net.n_params() == 8 * 64 * 9 + 64 + 2 * (64 * 64 * 9 + 64) + 64 * 6 * 9 + 6
    p = np.arange(net.n_params(), dtype=float)
    (W0, b0), *_ , (W3, b3) = net.unpack(p)
    assert W0.shape == (64, 8, 3, 3) and b0[0] == 8 * 64 * 9 and W3.shape == (6, 64, 3, 3)


def test_features_mask_block():
    L = 6
    rng = np.random.default_rng(1)
    th = rng.uniform(0, 2 * np.pi, 2 * L * L)
    X = net.features(th, L, 4, 5)
    bl = net.block_links(L, 4, 5)
    assert len(set(bl)) == 32
    assert X[6].sum() == 16 and X[7].sum() == 16
    th2 = th.copy()
    th2[bl] = rng.uniform(0, 2 * np.pi, 32)
    assert np.array_equal(net.features(th2, L, 4, 5), X)     # the proposal sees only the boundary


def test_gradient_finite_differences():
    L = 5
    rng = np.random.default_rng(2)
    params = small_params(3, 0.15)
    thetas = rng.uniform(0, 2 * np.pi, (2, 2 * L * L))
    blocks = [(0, 0), (3, 2)]
    loss, g = net.loss_and_grad(params, thetas, blocks, L)
    idx = rng.choice(net.n_params(), 40, replace=False)
    idx = np.concatenate([idx, [net.n_params() - 1, net.n_params() - 7, 8 * 64 * 9 + 3]])
    eps = 1e-6
    for i in idx:
        pp, pm = params.copy(), params.copy()
        pp[i] += eps
        pm[i] -= eps
        fd = (net.loss_and_grad(pp, thetas, blocks, L)[0] - net.loss_and_grad(pm, thetas, blocks, L)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


def test_log_q_matches_loss():
    L = 4
    rng = np.random.default_rng(4)
    params = small_params(5, 0.2)
    th = rng.uniform(0, 2 * np.pi, 2 * L * L)
    lq = net.log_q(params, th, L, 1, 2)
    loss, _ = net.loss_and_grad(params, th[None], [(1, 2)], L)
    assert abs(lq + loss) < 1e-12


@pytest.mark.parametrize("mu,rho", [(0.3, 0.1), (5.0, 0.8), (2.0, 0.95)])
def test_wrapped_cauchy_density_and_sampler(mu, rho):
    t = np.linspace(0, 2 * np.pi, 200001)
    f = np.exp(net.log_wc(t, mu, rho))
    assert abs(np.trapezoid(f, t) - 1.0) < 1e-6
    u = (np.arange(200000) + 0.5) / 200000
    s = net.sample_wc(mu, rho, u)
    assert np.all((s >= 0) & (s < 2 * np.pi))
    hist, edges = np.histogram(s, bins=40, range=(0, 2 * np.pi))
    cdf = lambda x: np.interp(x, t, np.concatenate([[0], np.cumsum(0.5 * (f[1:] + f[:-1]) * np.diff(t))]))
    want = (cdf(edges[1:]) - cdf(edges[:-1])) * len(s)
    assert np.abs(hist - want).max() <= 3 + 0.002 * len(s) / 40 + 0.01 * want.max()


def test_bf16_rounding():
    assert net.bf16(1.0) == 1.0
    assert net.bf16(1.0 + 2.0**-8) == 1.0                 # tie -> even (mantissa bit 0)
    assert net.bf16(1.0 + 3 * 2.0**-8) == 1.0 + 2.0**-6   # tie -> even (rounds up)
    assert net.bf16(1.0 + 2.0**-7) == 1.0 + 2.0**-7       # representable
    assert net.bf16(-2.5) == -2.5
    x = np.random.default_rng(0).normal(size=1000)
    assert np.all(np.abs(net.bf16(x) - x) <= 2.0**-8 * np.abs(x) * 1.0001)   # half an ulp of 7 bits


def test_quantised_network_is_the_plain_one_at_exact_values():
    """quant = identity gives the plain network; with BF16 rounding the loss moves by
    a rounding-sized amount only."""
    L = 4
    rng = np.random.default_rng(7)
    params = small_params(2, 0.1)
    th = rng.uniform(0, 2 * np.pi, (2, 2 * L * L))
    a = net.loss_and_grad(params, th, [(0, 0), (1, 3)], L)
    b = net.loss_and_grad(params, th, [(0, 0), (1, 3)], L, quant=lambda v: v)
    assert a[0] == b[0] and np.array_equal(a[1], b[1])
    c = net.loss_and_grad(params, th, [(0, 0), (1, 3)], L, quant=net.bf16)
    assert abs(c[0] - a[0]) < 1e-2 * abs(a[0])
