"""FP64 reference of the learned block proposal (test infrastructure).

The paper's method samples p(G) with local Metropolis moves (Sec. 5.1); the
learned proposal is an addition: a small convolutional network reads the links
outside a 4 x 4 block of sites and proposes new angles for the block's 32
links, and the move is accepted by exact Metropolis-Hastings against p(G).
This module is the plain, slow FP64 restatement used to check the GPU
network's forward pass, loss and gradients.

Network (shared convention with the CUDA kernels, each side its own code):

* Input, per site s = (x, y) of the L x L torus, 8 channels: cos, sin of the
  site's x-link angle; cos, sin of its y-link angle; cos, sin of the plaquette
  angle at s (theta1 + theta2 - theta3 - theta4, Sec. 2.3); a flag for "the
  x-link is in the block" and one for the y-link.  Angles of block links, and
  plaquettes that contain one, are zeroed: the proposal sees only the
  boundary, so its density is the same for the forward and reverse move.
* Block: sites ((bx + i) mod L, (by + j) mod L), i, j in 0..3; its links are
  the x- and y-links whose source site lies in the block (32 links).
* Layers: 3 x 3 convolutions with circular padding, 8 -> 64 -> 64 -> 64 -> 6
  channels, ReLU after the first three.  Parameters in one flat array, per
  layer W[co][ci][ky][kx] then bias[co]; input pixel of output (y, x) for
  tap (ky, kx) is ((y + ky - 1) mod L, (x + kx - 1) mod L).
* Head, per site: (a_x, b_x, z_x, a_y, b_y, z_y); for a block link in
  direction d: mu = atan2(b_d, a_d), rho = 0.95 sigmoid(z_d).  Proposal
  density: wrapped Cauchy f(t) = (1 - rho^2) / (2 pi (1 + rho^2 -
  2 rho cos(t - mu))); sample t = mu - log(rho) tan(pi (u - 1/2)) wrapped into
  [0, 2 pi).
* Training loss: mean over the batch of -sum over the 32 block links of
  log f(theta_link).

Optional `quant`: a rounding function applied where the GPU network stores
BF16 values (input features, weights, hidden activations after ReLU), so
that the GPU kernels can be compared with the same arithmetic up to FP32
accumulation; `bf16` below rounds to nearest even through FP32.

Pinned (tests/test_oracle_net.py): gradients against central finite
differences; the density integrates to 1; samples follow the density; the
BF16 rounding against hand-made bit patterns.
"""
from __future__ import annotations

import numpy as np

C_IN = 8
CH = 64
C_OUT = 6
LAYERS = [(C_IN, CH), (CH, CH), (CH, CH), (CH, C_OUT)]
RHO_MAX = 0.95
BLOCK = 4


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), via FP32, as float64."""
    a = np.asarray(x, dtype=np.float32).copy()
    u = a.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def n_params() -> int:
    return sum(co * ci * 9 + co for ci, co in LAYERS)


def unpack(params):
    out, k = [], 0
    for ci, co in LAYERS:
        W = params[k:k + co * ci * 9].reshape(co, ci, 3, 3)
        k += co * ci * 9
        b = params[k:k + co]
        k += co
        out.append((W, b))
    return out


def block_links(L: int, bx: int, by: int):
    """The 32 block links in order: block site (i, j) row-major, x then y."""
    out = []
    for j in range(BLOCK):
        for i in range(BLOCK):
            s = ((by + j) % L) * L + (bx + i) % L
            out += [2 * s, 2 * s + 1]
    return out


def features(theta: np.ndarray, L: int, bx: int, by: int) -> np.ndarray:
    """(C_IN, L, L) input for one configuration (angles, 2L^2) and block."""
    inb = np.zeros(2 * L * L, dtype=bool)
    inb[block_links(L, bx, by)] = True
    X = np.zeros((C_IN, L, L))
    for s in range(L * L):
        x, y = s % L, s // L
        lx, ly = 2 * s, 2 * s + 1
        if not inb[lx]:
            X[0, y, x], X[1, y, x] = np.cos(theta[lx]), np.sin(theta[lx])
        if not inb[ly]:
            X[2, y, x], X[3, y, x] = np.cos(theta[ly]), np.sin(theta[ly])
        sx, sy = y * L + (x + 1) % L, ((y + 1) % L) * L + x
        pl = (lx, 2 * sx + 1, 2 * sy, ly)
        if not any(inb[q] for q in pl):
            a = theta[pl[0]] + theta[pl[1]] - theta[pl[2]] - theta[pl[3]]
            X[4, y, x], X[5, y, x] = np.cos(a), np.sin(a)
        X[6, y, x] = float(inb[lx])
        X[7, y, x] = float(inb[ly])
    return X


def _shift(A, ky, kx):
    """A[..., (y + ky - 1) mod L, (x + kx - 1) mod L]."""
    return np.roll(A, shift=(1 - ky, 1 - kx), axis=(-2, -1))


def conv(X, W, b):
    """Circular 3x3 convolution of (B, ci, L, L) -> (B, co, L, L)."""
    out = np.broadcast_to(b[None, :, None, None], (X.shape[0], W.shape[0]) + X.shape[2:]).copy()
    for ky in range(3):
        for kx in range(3):
            out += np.einsum("oc,bcyx->boyx", W[:, :, ky, kx], _shift(X, ky, kx))
    return out


def conv_backward(X, W, dOut):
    dX = np.zeros_like(X)
    dW = np.zeros_like(W)
    for ky in range(3):
        for kx in range(3):
            Xs = _shift(X, ky, kx)
            dW[:, :, ky, kx] = np.einsum("boyx,bcyx->oc", dOut, Xs)
            # the tap read input pixel (y + ky - 1, x + kx - 1): send the gradient back
            g = np.einsum("oc,boyx->bcyx", W[:, :, ky, kx], dOut)
            dX += np.roll(g, shift=(ky - 1, kx - 1), axis=(-2, -1))
    return dX, dW, dOut.sum(axis=(0, 2, 3))


def forward(params, X, quant=None):
    """Head outputs (B, 6, L, L) and the per-layer activations."""
    q = quant if quant is not None else (lambda v: v)
    X = q(X)
    acts = [X]
    h = X
    layers = unpack(params)
    for k, (W, b) in enumerate(layers):
        z = conv(h, q(W), b)
        h = q(np.maximum(z, 0.0)) if k < len(layers) - 1 else z
        acts.append(h)
    return h, acts


def head_params(out, L, bx, by):
    """(mu, rho) of the 32 block links from head outputs (6, L, L)."""
    mus, rhos = [], []
    for j in range(BLOCK):
        for i in range(BLOCK):
            x, y = (bx + i) % L, (by + j) % L
            for d in range(2):
                a, bb, z = out[3 * d, y, x], out[3 * d + 1, y, x], out[3 * d + 2, y, x]
                mus.append(np.arctan2(bb, a))
                rhos.append(RHO_MAX / (1.0 + np.exp(-z)))
    return np.array(mus), np.array(rhos)


def log_wc(t, mu, rho):
    return np.log1p(-rho * rho) - np.log(2 * np.pi) - np.log(1.0 + rho * rho - 2.0 * rho * np.cos(t - mu))


def sample_wc(mu, rho, u):
    t = mu - np.log(rho) * np.tan(np.pi * (u - 0.5))
    return np.mod(t, 2 * np.pi)


def log_q(params, theta, L, bx, by, quant=None) -> float:
    """log density of the block links of `theta` under the proposal."""
    out, _ = forward(params, features(theta, L, bx, by)[None], quant)
    mu, rho = head_params(out[0], L, bx, by)
    t = theta[block_links(L, bx, by)]
    return float(np.sum(log_wc(t, mu, rho)))


def loss_and_grad(params, thetas, blocks, L, quant=None):
    """Mean over samples of -sum log f, and its gradient w.r.t. params.
    thetas: (B, 2L^2) angles; blocks: (B, 2) block origins."""
    B = len(thetas)
    X = np.stack([features(thetas[k], L, *blocks[k]) for k in range(B)])
    out, acts = forward(params, X, quant)
    q = quant if quant is not None else (lambda v: v)
    dOut = np.zeros_like(out)
    loss = 0.0
    for k in range(B):
        bx, by = blocks[k]
        links = block_links(L, bx, by)
        idx = 0
        for j in range(BLOCK):
            for i in range(BLOCK):
                x, y = (bx + i) % L, (by + j) % L
                for d in range(2):
                    a, bb, z = out[k, 3 * d, y, x], out[k, 3 * d + 1, y, x], out[k, 3 * d + 2, y, x]
                    sig = 1.0 / (1.0 + np.exp(-z))
                    rho = RHO_MAX * sig
                    mu = np.arctan2(bb, a)
                    t = thetas[k, links[idx]]
                    D = 1.0 + rho * rho - 2.0 * rho * np.cos(t - mu)
                    loss -= log_wc(t, mu, rho)
                    dmu = 2.0 * rho * np.sin(t - mu) / D
                    drho = -2.0 * rho / (1.0 - rho * rho) - (2.0 * rho - 2.0 * np.cos(t - mu)) / D
                    r2 = a * a + bb * bb
                    # d(-log f)/d(a, b, z) / B
                    dOut[k, 3 * d, y, x] += -(dmu * (-bb / r2)) / B
                    dOut[k, 3 * d + 1, y, x] += -(dmu * (a / r2)) / B
                    dOut[k, 3 * d + 2, y, x] += -(drho * RHO_MAX * sig * (1.0 - sig)) / B
                    idx += 1
    loss /= B
    grads = []
    layers = unpack(params)
    g = dOut
    for li in range(len(layers) - 1, -1, -1):
        W, b = layers[li]
        dX, dW, db = conv_backward(acts[li], q(W), g)
        grads.append((dW, db))
        if li > 0:
            g = dX * (acts[li] > 0.0)
    flat = []
    for dW, db in reversed(grads):
        flat += [dW.ravel(), db]
    return float(loss), np.concatenate(flat)
