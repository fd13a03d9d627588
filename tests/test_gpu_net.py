"""GPU proposal network (BF16 kernels) against the FP64 oracle network.

The oracle is evaluated with BF16 rounding at the points where the GPU stores
BF16 (features, weights, hidden activations), so the comparison isolates the
kernels (FP32 accumulation order) from the format; the gap between that and
the unrounded FP64 network is the format's own error and is reported by
bench-independent numbers in the test as a bound.  Training lowers the loss."""
import numpy as np
import pytest

from oracle import net as onet

pytestmark = pytest.mark.gpu


def make(L=6, seed=3):
    from paper_2412_01737_gb300 import Net
    return Net(0, L, seed)


def test_logq_matches_oracle():
    L = 6
    n = make(L)
    params = n.get_params().astype(np.float64)
    rng = np.random.default_rng(0)
    th = rng.uniform(0, 2 * np.pi, (5, 2 * L * L))
    bl = rng.integers(0, L, (5, 2))
    got = n.logq(th, bl)
    want = np.array([onet.log_q(params, th[k], L, *bl[k], quant=onet.bf16) for k in range(5)])
    exact = np.array([onet.log_q(params, th[k], L, *bl[k]) for k in range(5)])
    assert np.all(np.abs(got - want) <= 1e-3 * np.abs(want) + 1e-4), (got, want)
    assert np.all(np.abs(got - exact) <= 2e-2 * np.abs(exact) + 1e-3), (got, exact)
    n.close()


def test_gradient_matches_oracle():
    L = 5
    n = make(L, seed=9)
    rng = np.random.default_rng(1)
    # sharper outputs than the flat initial head, so every layer's gradient matters
    p = n.get_params()
    p[-(64 * 6 * 9 + 6):] *= 10.0
    n.set_params(p)
    params = n.get_params().astype(np.float64)
    th = rng.uniform(0, 2 * np.pi, (4, 2 * L * L))
    bl = rng.integers(0, L, (4, 2))
    loss, g = n.loss_grad(th, bl)
    lo, go = onet.loss_and_grad(params, th, [tuple(b) for b in bl], L, quant=onet.bf16)
    assert abs(loss - lo) <= 1e-3 * abs(lo)
    assert np.linalg.norm(g - go) <= 2e-2 * np.linalg.norm(go)
    # per layer, in norm and element by element: each entry within 5 % of its
    # oracle value plus 0.5 % of the layer's largest entry (FP32 accumulation
    # order moves activations across BF16 rounding boundaries now and then)
    k = 0
    for ci, co in onet.LAYERS:
        m = co * ci * 9 + co
        gl, ol = g[k:k + m], go[k:k + m]
        assert np.linalg.norm(gl - ol) <= 2e-2 * np.linalg.norm(ol) + 1e-6, (ci, co)
        bound = 5e-2 * np.abs(ol) + 5e-3 * np.abs(ol).max() + 1e-7
        bad = np.abs(gl - ol) > bound
        assert not bad.any(), (ci, co, int(bad.sum()), float((np.abs(gl - ol) / bound).max()))
        k += m
    # against the unrounded FP64 network: the BF16 format's own error
    le, ge = onet.loss_and_grad(params, th, [tuple(b) for b in bl], L)
    assert abs(loss - le) <= 2e-2 * abs(le)
    assert np.linalg.norm(g - ge) <= 0.15 * np.linalg.norm(ge)
    n.close()


def test_training_lowers_loss():
    import torch
    L = 6
    n = make(L, seed=4)
    rng = np.random.default_rng(2)
    # configurations concentrated near theta = 1.0: the proposal must learn mu and rho
    th = np.mod(1.0 + 0.1 * rng.standard_normal((64, 2 * L * L)), 2 * np.pi)
    dth = torch.from_numpy(th).cuda()
    losses = n.train(dth, 32, 200, 3e-3)
    assert losses[-20:].mean() < losses[:5].mean() - 20.0, (losses[:5], losses[-20:])
    n.close()
