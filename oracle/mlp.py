"""Network of the learned boundary closure, float64 (test infrastructure).

A 12 -> 64 -> 64 -> 5 multilayer perceptron with tanh hidden layers; the
closure it serves maps the interior trace at an outer-face node to a
correction of the characteristic ghost state. Written out layer by layer:

    h1 = tanh(x W1 + b1),  h2 = tanh(h1 W2 + b2),  y = h2 W3 + b3
    loss = (1/N) sum_n sum_o (y_no - t_no)^2

with the backward pass obtained by the chain rule, and Adam (Kingma & Ba,
2015) with beta1 = 0.9, beta2 = 0.999, eps = 1e-8. Parameters are one flat
vector packed as W1[12][64], b1[64], W2[64][64], b2[64], W3[64][5], b3[5]
(input index first).

Features of a face node (interior perturbation trace q', outward normal n,
position x, scale R, memory psi) come from what the interior determines
there: the outgoing acoustic invariant w_out = p' + rho0 c0 u.n, the entropy
mode, the tangential velocity and the node's memory psi of past outgoing
waves (``oracle.euler_dg.memory_rate``), each divided by the amplitude
s = (|w_out| + |psi|) / (rho0 c0^2) + 1e-12 (see ``features``). Output 0 is
the incoming invariant the closure sets, relative to the memory psi (the
spherical-wave value), in units of rho0 c0^2 s; the closure itself (bounded,
invariant by invariant) is ``oracle.euler_dg.ghost_learned``.

Parity status: pinned (tests/test_oracle_mlp.py: central finite differences
of the loss, closed forms at zero weights, Adam's first step, the feature
definition on a hand-computed state, invariance of the features under a
change of the incoming invariant).
"""
from __future__ import annotations

import numpy as np

N_IN, N_H, N_OUT = 12, 64, 5
SIZES = [("W1", (N_IN, N_H)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)),
         ("W3", (N_H, N_OUT)), ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(w):
    out, o = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = np.asarray(w[o:o + k], dtype=np.float64).reshape(shape)
        o += k
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SIZES])


def init_params(seed=0, scale=1.0):
    """Seeded Glorot-uniform weights and zero biases."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shape in SIZES:
        if name.startswith("W"):
            lim = scale * np.sqrt(6.0 / (shape[0] + shape[1]))
            p[name] = rng.uniform(-lim, lim, size=shape)
        else:
            p[name] = np.zeros(shape)
    return pack(p)


def forward(w, X):
    p = unpack(w)
    h1 = np.tanh(X @ p["W1"] + p["b1"])
    h2 = np.tanh(h1 @ p["W2"] + p["b2"])
    return h2 @ p["W3"] + p["b3"], (h1, h2)


def loss_and_grad(w, X, T):
    """Mean (over samples) of the summed squared output error, and its gradient."""
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    p = unpack(w)
    N = X.shape[0]
    y, (h1, h2) = forward(w, X)
    d = y - T
    loss = np.sum(d * d) / N
    dy = 2.0 * d / N
    g = {"W3": h2.T @ dy, "b3": dy.sum(axis=0)}
    dz2 = (dy @ p["W3"].T) * (1.0 - h2 * h2)
    g["W2"] = h1.T @ dz2
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ p["W2"].T) * (1.0 - h1 * h1)
    g["W1"] = X.T @ dz1
    g["b1"] = dz1.sum(axis=0)
    return loss, pack(g)


def adam(w, X, T, iters, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """Full-batch Adam; returns (w, loss before each step)."""
    w = np.array(w, dtype=np.float64)
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    hist = []
    for t in range(1, iters + 1):
        loss, g = loss_and_grad(w, X, T)
        hist.append(loss)
        m = beta1 * m + (1 - beta1) * g
        v = beta2 * v + (1 - beta2) * g * g
        w = w - lr * (m / (1 - beta1 ** t)) / (np.sqrt(v / (1 - beta2 ** t)) + eps)
    return w, np.array(hist)


# ------------------------------------------------------------- the closure

def normalise(q, rho0, c0):
    """z of perturbation states q[..., 5]."""
    z = np.array(q, dtype=np.float64, copy=True)
    z[..., 0] /= rho0
    z[..., 1:4] /= rho0 * c0
    z[..., 4] /= rho0 * c0 * c0
    return z


def denormalise(z, rho0, c0):
    q = np.array(z, dtype=np.float64, copy=True)
    q[..., 0] *= rho0
    q[..., 1:4] *= rho0 * c0
    q[..., 4] *= rho0 * c0 * c0
    return q


def features(qp, n, x, psi, gas, radius):
    """Features [..., 12] and amplitude s [...] of perturbation traces qp[..., 5]
    with memory psi[...]:
    (w_out / (rho0 c0^2 s), (rho' - p'/c0^2) / (rho0 s), u_t / (c0 s), n, x / R,
    psi / (rho0 c0^2 s)) with w_out = p' + rho0 c0 u.n and
    s = (|w_out| + |psi|) / (rho0 c0^2) + 1e-12."""
    rho = gas.rho0 + qp[..., 0]
    pp = (gas.gamma - 1.0) * (qp[..., 4] - 0.5 * np.sum(qp[..., 1:4] ** 2, axis=-1) / rho)
    u = qp[..., 1:4] / rho[..., None]
    un = np.sum(u * n, axis=-1)
    pref = gas.rho0 * gas.c0 ** 2
    wout = pp + gas.rho0 * gas.c0 * un
    s = (np.abs(wout) + np.abs(psi)) / pref + 1e-12
    ent = (qp[..., 0] - pp / gas.c0 ** 2) / (gas.rho0 * s)
    ut = (u - un[..., None] * n) / (gas.c0 * s[..., None])
    f = np.concatenate([(wout / (pref * s))[..., None], ent[..., None], ut, n, x / radius,
                        (psi / (pref * s))[..., None]], axis=-1)
    return f, s
