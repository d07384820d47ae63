"""FP64 oracle of the learned-CPML network (test infrastructure).

The paper fixes the CPML of Sec. 3.2 (polynomial grading, Tab. 2) and names
learned discretisations only as future work (Sec. 7).  The learned form here
replaces the polynomial grading of a thin layer by a small network that maps
per-cell features to (sigma, kappa, alpha); everything downstream of
(sigma, kappa, alpha) is the paper's CPML (Sec. 3.2 coefficients b, a, 1/kappa).

Network: 4 -> 64 -> 64 -> 3, tanh hidden activations, outputs
  sigma = sigma_scale * softplus(o_0)
  kappa = 1 + softplus(o_1)
  alpha = alpha_scale * softplus(o_2)
so that sigma >= 0, kappa >= 1, alpha >= 0.

Parameter vector layout (4675 values, row-major):
  W1 [64, 4], b1 [64], W2 [64, 64], b2 [64], W3 [3, 64], b3 [3].

Features of layer cell j (j = 0 outermost, depth index into an L-cell layer):
  [rho_j = (L - j)/L, L / L_ref, f0 h / c, c dt / h].
"""
from __future__ import annotations

import numpy as np

from . import oracle as O

SIZES = [(64, 4), (64,), (64, 64), (64,), (3, 64), (3,)]
NPARAM = int(sum(np.prod(s) for s in SIZES))


def unpack(theta):
    out, o = [], 0
    for s in SIZES:
        n = int(np.prod(s))
        out.append(np.asarray(theta[o:o + n], dtype=np.float64).reshape(s))
        o += n
    return out


def softplus(x):
    return np.logaddexp(0.0, x)


def sigmoid(x):
    return 0.5 * (1.0 + np.tanh(0.5 * x))


def forward(theta, X, sigma_scale, alpha_scale):
    """X [n, 4] -> (out [n, 3] = sigma, kappa, alpha; cache)."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1.T + b1
    h1 = np.tanh(z1)
    z2 = h1 @ W2.T + b2
    h2 = np.tanh(z2)
    o = h2 @ W3.T + b3
    sp = softplus(o)
    out = np.stack([sigma_scale * sp[:, 0], 1.0 + sp[:, 1], alpha_scale * sp[:, 2]], axis=1)
    return out, (X, h1, h2, o)


def backward(theta, cache, gout, sigma_scale, alpha_scale):
    """dJ/dtheta from dJ/d(sigma, kappa, alpha) per sample (gout [n, 3])."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    X, h1, h2, o = cache
    scale = np.array([sigma_scale, 1.0, alpha_scale])
    go = gout * scale[None, :] * sigmoid(o)          # d softplus = sigmoid
    gW3 = go.T @ h2
    gb3 = go.sum(0)
    gh2 = go @ W3
    gz2 = gh2 * (1.0 - h2 * h2)
    gW2 = gz2.T @ h1
    gb2 = gz2.sum(0)
    gh1 = gz2 @ W2
    gz1 = gh1 * (1.0 - h1 * h1)
    gW1 = gz1.T @ X
    gb1 = gz1.sum(0)
    return np.concatenate([g.ravel() for g in (gW1, gb1, gW2, gb2, gW3, gb3)])


def adam_step(theta, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba): returns new (theta, m, v); t counts from 1."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mhat = m / (1 - beta1 ** t)
    vhat = v / (1 - beta2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def init_params(seed: int, scale1=0.5, scale2=0.2, scale3=0.1):
    """Seeded initial weights (normal, fixed scales), zero biases."""
    rng = np.random.default_rng(seed)
    W1 = scale1 * rng.standard_normal((64, 4))
    W2 = scale2 * rng.standard_normal((64, 64))
    W3 = scale3 * rng.standard_normal((3, 64))
    return np.concatenate([W1.ravel(), np.zeros(64), W2.ravel(), np.zeros(64),
                           W3.ravel(), np.zeros(3)])


def features(L, L_ref, f0, h, c, dt):
    """[n = L, 4] feature rows of the layer cells j = 0..L-1 (outermost first)."""
    j = np.arange(L)
    rho = (L - j) / L
    return np.stack([rho, np.full(L, L / L_ref), np.full(L, f0 * h / c),
                     np.full(L, c * dt / h)], axis=1)


def coefficient_jacobian(sigma, kappa, alpha, dt):
    """b, a, kinv of Sec. 3.2 and their partial derivatives with respect to
    (sigma, kappa, alpha), analytically.  Returns (b, a, kinv, J) with
    J[..., k, m] = d coef_k / d param_m, coef = (b, a, kinv),
    param = (sigma, kappa, alpha)."""
    sigma, kappa, alpha = (np.asarray(x, dtype=np.float64) for x in (sigma, kappa, alpha))
    b = np.exp(-(sigma / kappa + alpha) * dt)
    db = np.stack([-dt / kappa * b, dt * sigma / kappa ** 2 * b, -dt * b], axis=-1)
    D = kappa * sigma + kappa ** 2 * alpha
    a = sigma * (b - 1.0) / D
    dD = np.stack([kappa, sigma + 2 * kappa * alpha, kappa ** 2], axis=-1)
    num = sigma * (b - 1.0)
    dnum = np.stack([(b - 1.0) + sigma * db[..., 0], sigma * db[..., 1], sigma * db[..., 2]],
                    axis=-1)
    da = dnum / D[..., None] - num[..., None] * dD / (D ** 2)[..., None]
    kinv = 1.0 / kappa
    dk = np.stack([np.zeros_like(kappa), -1.0 / kappa ** 2, np.zeros_like(kappa)], axis=-1)
    return b, a, kinv, np.stack([db, da, dk], axis=-2)


def learned_profiles(shape, L, ska, dt):
    """Per-axis profiles (slab, b, a, kinv) of a grid with L cells on every
    face from per-cell (sigma, kappa, alpha) ska[L, 3], cell j on node j of the
    low face and node n-1-j of the high face of each axis."""
    nz, ny, nx = shape
    b, a, kinv, _ = coefficient_jacobian(ska[:, 0], ska[:, 1], ska[:, 2], dt)
    prof = []
    for n in (nx, ny, nz):
        pr = dict(slab=np.zeros(n, np.uint8), b=np.zeros(n), a=np.zeros(n), kinv=np.ones(n))
        for j in range(L):
            for i in (j, n - 1 - j):
                pr["slab"][i] = 1
                pr["b"][i], pr["a"][i], pr["kinv"][i] = b[j], a[j], kinv[j]
        prof.append(pr)
    return prof


def ska_gradient_from_profile_gradient(shape, L, ska, dt, gprof):
    """Chain rule: dJ/d(sigma, kappa, alpha) per cell from dJ/d(b, a, kinv)
    per axis and node (gprof [3, 3, nmax]), summing the six nodes that share
    a cell."""
    nz, ny, nx = shape
    _, _, _, Jc = coefficient_jacobian(ska[:, 0], ska[:, 1], ska[:, 2], dt)
    g = np.zeros((L, 3))
    for d, n in enumerate((nx, ny, nz)):
        for j in range(L):
            for i in (j, n - 1 - j):
                g[j] += gprof[d, :, i] @ Jc[j]
    return g


def learned_misfit_gradient(theta, shape, L, dt, h, K, feats, sigma_scale, alpha_scale,
                            shots, nt, checkpoint_every=10):
    """J = sum over shots of 1/2 ||traces - reference||^2 with the learned
    layer, and dJ/dtheta.  shots: list of (src, wavelet, rec, reference)."""
    ska, cache = forward(theta, feats, sigma_scale, alpha_scale)
    prof = learned_profiles(shape, L, ska, dt)
    g = O.Grid(K, h, dt, prof)
    J = 0.0
    gprof = np.zeros((3, 3, max(shape)))
    for src, wav, rec, ref in shots:
        Js, _, gp, _ = O.misfit_gradient(g, nt, src, wav, rec, ref, checkpoint_every,
                                         want_profiles=True)
        J += Js
        gprof += gp
    gska = ska_gradient_from_profile_gradient(shape, L, ska, dt, gprof)
    return J, backward(theta, cache, gska, sigma_scale, alpha_scale), ska
