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

Standardisation over a training set of rows D (n x 32) and targets t (n):
    mu_j = mean_p D[p, j],  sd_j = sqrt(sum_p (D[p, j] - mu_j)^2 / (n - 1)),
    inv_sd_j = 1/sd_j (0 when sd_j <= 1e-6: a constant feature is switched off),
    t_shift = mean t,  t_scale = sqrt(sum (t - t_shift)^2 / (n - 1)) (1 when that is 0),
    t_norm = (t - t_shift) / t_scale.
Training target per domain point: dV = V_in(converged) - V_start.
Correction: dV(p) = y(D[p]) t_scale + t_shift.

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


SD_FLOOR = 1e-6


def standardise(D, t):
    """(mu, inv_sd, t_shift, t_scale, t_norm) of a training set (see the module docstring)."""
    D = np.asarray(D, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    n = len(t)
    mu = D.sum(0) / n
    sd = np.sqrt(((D - mu) ** 2).sum(0) / (n - 1))
    inv_sd = np.where(sd > SD_FLOOR, 1.0 / np.where(sd > SD_FLOOR, sd, 1.0), 0.0)
    t_shift = t.sum() / n
    t_scale = math.sqrt(((t - t_shift) ** 2).sum() / (n - 1))
    if t_scale == 0.0:
        t_scale = 1.0
    return mu, inv_sd, t_shift, t_scale, (t - t_shift) / t_scale


def training_target(v_in, v_start):
    """dV = V_in(converged) - V_start per domain point."""
    return np.asarray(v_in, dtype=np.float64) - np.asarray(v_start, dtype=np.float64)


def correction(params, mu, inv_sd, t_shift, t_scale, D):
    """dV per row of D: the network on the standardised descriptors, de-standardised."""
    x = (np.asarray(D, dtype=np.float64) - mu) * inv_sd
    y, _ = forward(params, x)
    return y * t_scale + t_shift
