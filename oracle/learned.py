"""Learned SCF start (oracle, float64) -- test infrastructure only.

The paper has no learned component; this is the reference for the project's own
learned starting potential: a per-grid-point correction dV of the superposition start,
predicted by a small multilayer perceptron from radial descriptors of the surrounding
atoms.  Everything here is plain numpy in float64 and follows the definitions below
step by step.

Descriptors (32 per grid point p): for the two species s (Si, H) and the 16 radial
centres c_q = q * r_c / 15 (q = 0..15, r_c = 8 bohr),
    D[p, 16 s + q] = sum over atoms a of species s with r = |p - R_a| < r_c of
                     exp(-(r - c_q)^2 / (2 sigma^2)) * (1 + cos(pi r / r_c)) / 2,
    sigma = r_c / 15 (the centre spacing).

Network (inputs standardised, x = (D - mu) / sd):
    h1 = tanh(x W1 + b1)      W1: 32 x 128
    h2 = tanh(h1 W2 + b2)     W2: 128 x 128
    y  = h2 w3 + b3           w3: 128
Loss: L = mean over the batch of (y - t)^2 (t: standardised target).
Adam (Kingma & Ba 2015): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
    p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
"""
from __future__ import annotations

import math

import numpy as np

N_RADIAL = 16
R_CUT = 8.0
DESC_Z = (14, 1)
N_IN, N_HID = 32, 128


def radial_centres():
    return np.arange(N_RADIAL, dtype=np.float64) * (R_CUT / (N_RADIAL - 1))


def descriptors(points, atom_pos, atom_z):
    """(n_points, 32) radial descriptors (loop over atoms; float64)."""
    points = np.asarray(points, dtype=np.float64)
    c = radial_centres()
    sigma = R_CUT / (N_RADIAL - 1)
    D = np.zeros((len(points), N_IN))
    for pos, z in zip(np.asarray(atom_pos, dtype=np.float64), atom_z):
        s = DESC_Z.index(int(z))
        d = points - pos
        r = np.sqrt((d * d).sum(1))
        near = r < R_CUT
        rn = r[near]
        fc = 0.5 * (1.0 + np.cos(math.pi * rn / R_CUT))
        D[np.ix_(near, np.arange(16 * s, 16 * s + 16))] += (
            np.exp(-((rn[:, None] - c[None, :]) ** 2) / (2.0 * sigma * sigma)) * fc[:, None])
    return D


def init_params(seed: int):
    """Glorot-uniform weights, zero biases (seeded)."""
    rng = np.random.default_rng(seed)

    def glorot(fan_in, fan_out, shape):
        lim = math.sqrt(6.0 / (fan_in + fan_out))
        return rng.uniform(-lim, lim, shape)

    return {"W1": glorot(N_IN, N_HID, (N_IN, N_HID)), "b1": np.zeros(N_HID),
            "W2": glorot(N_HID, N_HID, (N_HID, N_HID)), "b2": np.zeros(N_HID),
            "w3": glorot(N_HID, 1, (N_HID,)), "b3": np.zeros(1)}


def forward(params, x):
    h1 = np.tanh(x @ params["W1"] + params["b1"])
    h2 = np.tanh(h1 @ params["W2"] + params["b2"])
    y = h2 @ params["w3"] + params["b3"][0]
    return y, (x, h1, h2)


def loss_and_grad(params, x, t):
    """Mean squared error and its gradient (backpropagation through the three layers)."""
    y, (x, h1, h2) = forward(params, x)
    n = len(t)
    r = y - t
    loss = float(np.mean(r * r))
    dy = 2.0 * r / n
    g = {"w3": h2.T @ dy, "b3": np.array([dy.sum()])}
    g2 = np.outer(dy, params["w3"]) * (1.0 - h2 * h2)
    g["W2"] = h1.T @ g2
    g["b2"] = g2.sum(0)
    g1 = (g2 @ params["W2"].T) * (1.0 - h1 * h1)
    g["W1"] = x.T @ g1
    g["b1"] = g1.sum(0)
    return loss, g


def adam_step(params, grads, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step number t >= 1) of every array in params, in place."""
    for key in params:
        m[key] = beta1 * m[key] + (1.0 - beta1) * grads[key]
        v[key] = beta2 * v[key] + (1.0 - beta2) * grads[key] ** 2
        mh = m[key] / (1.0 - beta1 ** t)
        vh = v[key] / (1.0 - beta2 ** t)
        params[key] = params[key] - lr * mh / (np.sqrt(vh) + eps)
    return params, m, v


def pack(params):
    """Flat parameter vector in the library's order: W1 (row-major 32x128), b1, W2
    (row-major 128x128), b2, w3, b3."""
    return np.concatenate([params["W1"].ravel(), params["b1"], params["W2"].ravel(), params["b2"],
                           params["w3"], params["b3"]])


def unpack(flat):
    flat = np.asarray(flat, dtype=np.float64)
    o = 0
    out = {}
    for key, shape in (("W1", (N_IN, N_HID)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
                       ("w3", (N_HID,)), ("b3", (1,))):
        size = int(np.prod(shape))
        out[key] = flat[o:o + size].reshape(shape)
        o += size
    return out


N_PARAMS = N_IN * N_HID + N_HID + N_HID * N_HID + N_HID + N_HID + 1
