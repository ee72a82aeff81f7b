"""Oracle: FP64 reference of the learned coarse correction's network.

Test infrastructure only. The paper has no learned component; this is the
plain FP64 definition of the three-layer ReLU network that maps a normalised
restricted residual x = P^T r1 / ||P^T r1|| (length k) to a coarse
correction: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), o = W3 h2 + b3, with
the squared-error loss 0.5/B sum ||o - t||^2 over a batch of B rows, its
gradients by the chain rule, and one Adam step (Kingma & Ba, ICLR 2015).
Row-major batches: X is (B, k), W1 is (H, k), W2 is (H, H), W3 is (k, H).

A metric W (symmetric positive definite k x k, e.g. the coarse operator A_c)
weights the loss: 0.5/B sum (o - t)^T W (o - t); the output gradient is then
W (o - t) / B per row. With W = A_c the error of a coarse correction is
measured in the energy norm of the coarse space, the norm in which the
Galerkin coarse solve is optimal.
"""
from __future__ import annotations

import numpy as np


def init_params(k, hidden, seed_uniforms):
    """He-uniform initial weights from a supplied stream of uniforms in [0,1);
    biases zero. seed_uniforms(n) must return n uniforms."""
    def he(fan_out, fan_in):
        bound = np.sqrt(6.0 / fan_in)
        return (2.0 * seed_uniforms(fan_out * fan_in) - 1.0).reshape(fan_out, fan_in) * bound
    return {"W1": he(hidden, k), "b1": np.zeros(hidden),
            "W2": he(hidden, hidden), "b2": np.zeros(hidden),
            "W3": he(k, hidden), "b3": np.zeros(k)}


def forward(p, X):
    a1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    o = h2 @ p["W3"].T + p["b3"]
    return o, (X, a1, h1, a2, h2)


def loss(p, X, T, W=None):
    o, _ = forward(p, X)
    D = o - T
    if W is None:
        return 0.5 * np.sum(D ** 2) / X.shape[0]
    return 0.5 * np.sum((D @ W) * D) / X.shape[0]


def backward(p, X, T, W=None):
    """Gradients of loss() with respect to every parameter."""
    o, (X, a1, h1, a2, h2) = forward(p, X)
    B = X.shape[0]
    do = (o - T) / B
    if W is not None:
        do = do @ W
    g = {"W3": do.T @ h2, "b3": do.sum(0)}
    dh2 = do @ p["W3"]
    da2 = dh2 * (a2 > 0.0)
    g["W2"] = da2.T @ h1
    g["b2"] = da2.sum(0)
    dh1 = da2 @ p["W2"]
    da1 = dh1 * (a1 > 0.0)
    g["W1"] = da1.T @ X
    g["b1"] = da1.sum(0)
    return g


def adam_step(p, g, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update in place; state holds m, v and the step count t."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for name in p:
        m = state.setdefault("m_" + name, np.zeros_like(p[name]))
        v = state.setdefault("v_" + name, np.zeros_like(p[name]))
        m *= b1
        m += (1.0 - b1) * g[name]
        v *= b2
        v += (1.0 - b2) * g[name] ** 2
        mhat = m / (1.0 - b1 ** t)
        vhat = v / (1.0 - b2 ** t)
        p[name] -= lr * mhat / (np.sqrt(vhat) + eps)


def coarse_correction(p, rc):
    """e_c = ||rc|| * net(rc / ||rc||): positively homogeneous in rc."""
    nrm = float(np.linalg.norm(rc))
    if nrm == 0.0:
        return np.zeros_like(rc)
    o, _ = forward(p, (rc / nrm)[None, :])
    return nrm * o[0]
