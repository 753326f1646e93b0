"""Pins of the learned-start oracle (oracle/learned.py) against closed forms, invariances
and finite differences."""
import math

import numpy as np

from oracle import learned as L


def test_descriptor_single_atom_closed_form():
    c = L.radial_centres()
    sigma = L.R_CUT / 15
    u = np.array([0.6, -0.8, 0.0])
    for s, z in enumerate(L.DESC_Z):
        for q in (0, 3, 15):
            r = c[q] * 0.999 if q == 15 else c[q]          # inside the cutoff
            D = L.descriptors(np.array([[0.2, 0.1, -0.3]]), np.array([[0.2, 0.1, -0.3]]) + r * u, [z])[0]
            fc = 0.5 * (1 + math.cos(math.pi * r / L.R_CUT))
            # the Gaussian centred on this distance is at its peak; its neighbours are
            # one spacing away: exp(-1/2)
            assert abs(D[16 * s + q] - math.exp(-((r - c[q]) ** 2) / (2 * sigma ** 2)) * fc) < 1e-15
            if q == 3:
                assert abs(D[16 * s + 3] - fc) < 1e-15
                assert abs(D[16 * s + 2] - math.exp(-0.5) * fc) < 1e-15
            assert np.all(D[16 * (1 - s):16 * (1 - s) + 16] == 0)


def test_descriptor_cutoff_invariance_additivity():
    rng = np.random.default_rng(1)
    atoms = rng.uniform(-6, 6, (12, 3))
    z = np.array([14, 1] * 6)
    pts = rng.uniform(-3, 3, (20, 3))
    D = L.descriptors(pts, atoms, z)
    # rotation of everything about a point leaves that point's descriptor unchanged
    from workloads.cluster import random_rotation
    R = random_rotation(7)
    p0 = pts[:1]
    Dr = L.descriptors(p0, (atoms - p0) @ R.T + p0, z)
    assert np.allclose(Dr, D[:1], atol=1e-13)
    # additivity over atom subsets
    Da = L.descriptors(pts, atoms[:5], z[:5]) + L.descriptors(pts, atoms[5:], z[5:])
    assert np.allclose(Da, D, atol=1e-14)
    # atoms at or beyond the cutoff contribute nothing; continuity just inside
    far = L.descriptors(pts[:1], pts[:1] + np.array([[L.R_CUT, 0, 0]]), [14])
    assert np.all(far == 0)
    near = L.descriptors(pts[:1], pts[:1] + np.array([[L.R_CUT - 1e-6, 0, 0]]), [14])
    assert np.max(np.abs(near)) < 1e-10


def test_network_zero_weights_and_parameter_layout():
    p = L.init_params(0)
    for k in p:
        p[k] = np.zeros_like(p[k])
    p["b3"][0] = 0.37
    y, _ = L.forward(p, np.random.default_rng(0).standard_normal((5, 32)))
    assert np.all(y == 0.37)
    q = L.init_params(3)
    flat = L.pack(q)
    assert flat.size == L.N_PARAMS == 32 * 128 + 128 + 128 * 128 + 128 + 128 + 1
    back = L.unpack(flat)
    assert all(np.array_equal(back[k], q[k]) for k in q)


def test_forward_single_path_closed_form():
    """One non-zero weight per layer (input i -> hidden j -> hidden k -> output) gives
    y = w3_k tanh(W2_jk tanh(W1_ij x_i + b1_j) + b2_k) + b3 exactly: every other hidden
    unit sees tanh(0) = 0.  A different activation, a transposed W2 (j != k) or a dropped
    bias changes y."""
    p = L.init_params(0)
    for key in p:
        p[key] = np.zeros_like(p[key])
    i, j, k = 5, 17, 90
    p["W1"][i, j], p["b1"][j] = 0.8, -0.3
    p["W2"][j, k], p["b2"][k] = -1.7, 0.25
    p["w3"][k], p["b3"][0] = 2.5, 0.1
    x = np.zeros((4, 32))
    x[:, i] = [-2.0, -0.4, 0.0, 1.3]
    x[:, 3] = 9.0                      # an input with no path to the output
    y, (_, h1, h2) = L.forward(p, x)
    expect = 2.5 * np.tanh(-1.7 * np.tanh(0.8 * x[:, i] - 0.3) + 0.25) + 0.1
    assert np.allclose(y, expect, rtol=0, atol=1e-15)
    assert np.count_nonzero(h1) == 4 and np.count_nonzero(h2) == 4


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(4)
    p = L.init_params(11)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.standard_normal(p[k].shape) * 0.1
    x = rng.standard_normal((7, 32))
    t = rng.standard_normal(7)
    _, g = L.loss_and_grad(p, x, t)
    flat = L.pack(p)
    gflat = L.pack(g)
    idx = rng.choice(flat.size, 60, replace=False)
    idx = np.concatenate([idx, [L.N_PARAMS - 1, 0, 32 * 128 + 5]])
    for i in idx:
        e = np.zeros_like(flat)
        e[i] = 1e-6
        lp, _ = L.loss_and_grad(L.unpack(flat + e), x, t)
        lm, _ = L.loss_and_grad(L.unpack(flat - e), x, t)
        fd = (lp - lm) / 2e-6
        assert abs(fd - gflat[i]) < 1e-7 * max(1.0, abs(fd)), (i, fd, gflat[i])


def test_adam_first_step_is_signed_learning_rate():
    p = {"a": np.array([1.0, -2.0, 3.0])}
    g = {"a": np.array([0.5, -4.0, 0.0])}
    m = {"a": np.zeros(3)}
    v = {"a": np.zeros(3)}
    p, m, v = L.adam_step(p, g, m, v, 1, lr=0.01)
    # m_hat = g, v_hat = g^2: the step is lr * g / (|g| + eps)
    assert np.allclose(p["a"], [1.0 - 0.01 * 0.5 / (0.5 + 1e-8), -2.0 + 0.01 * 4.0 / (4.0 + 1e-8), 3.0], atol=1e-15)


def test_standardise_closed_form_and_invariants():
    """Two rows (0, 2) give mean 1 and unbiased sd sqrt(2); a constant feature gets
    inv_sd 0; the standardised set has mean 0 and unbiased variance 1 per live feature; a
    biased (1/n) variance or a missing floor fails."""
    D = np.zeros((2, 32))
    D[:, 0] = [0.0, 2.0]
    D[:, 1] = 5.0
    mu, inv_sd, ts, sc, tn = L.standardise(D, np.array([1.0, 3.0]))
    assert mu[0] == 1.0 and abs(inv_sd[0] - 1.0 / math.sqrt(2.0)) < 1e-15 and inv_sd[1] == 0.0
    assert ts == 2.0 and abs(sc - math.sqrt(2.0)) < 1e-15
    assert np.allclose(tn, [-1.0 / math.sqrt(2.0), 1.0 / math.sqrt(2.0)], atol=1e-15)
    rng = np.random.default_rng(4)
    D = rng.uniform(0, 3, (500, 32))
    D[:, 7] = 0.25
    t = rng.standard_normal(500) * 0.3 + 0.1
    mu, inv_sd, ts, sc, tn = L.standardise(D, t)
    X = (D - mu) * inv_sd
    live = np.arange(32) != 7
    assert np.allclose(X[:, live].mean(0), 0.0, atol=1e-12) and np.allclose(X[:, live].var(0, ddof=1), 1.0)
    assert np.all(X[:, 7] == 0) and abs(tn.mean()) < 1e-12 and abs(tn.var(ddof=1) - 1.0) < 1e-12
    # constant target: scale 1
    assert L.standardise(D, np.full(500, 0.4))[3] == 1.0


def test_correction_is_affine_in_the_network_output():
    p = L.init_params(2)
    rng = np.random.default_rng(6)
    D = rng.uniform(0, 2, (9, 32))
    mu, inv_sd = D.mean(0), np.full(32, 0.7)
    y, _ = L.forward(p, (D - mu) * inv_sd)
    assert np.allclose(L.correction(p, mu, inv_sd, 0.3, 2.5, D), 2.5 * y + 0.3, rtol=0, atol=1e-14)
    assert np.array_equal(L.training_target([1.0, 2.0], [0.5, 3.0]), [0.5, -1.0])
