"""Pins of the oracle's grid construction against brute-force enumeration."""
import numpy as np

from oracle.grid import box_grid, sphere_grid


def test_sphere_matches_bruteforce():
    R, h = 3.1, 0.7
    n = int(R / h) + 2
    pts = []
    for k in range(-n, n + 1):
        for j in range(-n, n + 1):
            for i in range(-n, n + 1):
                if (i * i + j * j + k * k) * h * h <= R * R * (1 + 1e-12):
                    pts.append((i, j, k))
    g = sphere_grid((0.0, 0.0, 0.0), R, h)
    assert [tuple(x) for x in g.ijk.tolist()] == pts  # same set, same (k, j, i) order


def test_sphere_volume_and_lookup():
    R, h = 9.0, 0.5
    g = sphere_grid((1.0, -2.0, 0.5), R, h)
    vol = 4.0 / 3.0 * np.pi * (R / h) ** 3
    assert abs(g.n - vol) / vol < 0.01
    rng = np.random.default_rng(0)
    sel = rng.integers(0, g.n, 200)
    assert np.array_equal(g.index_of(g.ijk[sel]), sel)
    far = np.array([[100, 0, 0], [0, 0, 19], [13, 13, 0]])
    assert np.all(g.index_of(far) == -1)
    assert g.index_of(np.array([[0, 0, 18], [18, 0, 0]])).min() >= 0   # ties are inclusive


def test_box_grid():
    g = box_grid(3, 4, 5, 0.5)
    assert g.n == 60
    assert tuple(g.ijk[1]) == (1, 0, 0) and tuple(g.ijk[3]) == (0, 1, 0) and tuple(g.ijk[12]) == (0, 0, 1)
