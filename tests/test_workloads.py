"""Pins of the shared input generators: cluster geometry, occupation counts, RNG."""
import os

import numpy as np
import pytest

from workloads import (WORKLOADS, n_electrons, n_occupied, normal_entries, random_block_lex,
                       silicon_cluster)
from workloads.cluster import ANG2BOHR

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_nanoclusters.txt")


def test_diamond_shells():
    # neighbour shells of a diamond site at a = 5.43 A: 4, 12, 12, 6, 12 atoms
    pos, z = silicon_cluster(6.0)
    si = pos[z == 14] / ANG2BOHR
    r = np.sqrt((si ** 2).sum(1))
    shells = [(2.351, 4), (3.840, 12), (4.503, 12), (5.430, 6)]
    for d, n in shells:
        assert np.count_nonzero(np.abs(r - d) < 2e-3) == n


def test_si35h36():
    pos, z = silicon_cluster(5.7)
    assert np.count_nonzero(z == 14) == 35 and np.count_nonzero(z == 1) == 36
    assert np.allclose(pos[0], 0.0)
    assert n_electrons(z) == 176 and n_occupied(z) == 88
    # every H sits 1.48 A from exactly one Si
    si, h = pos[z == 14], pos[z == 1]
    d = np.sqrt(((h[:, None, :] - si[None, :, :]) ** 2).sum(-1)) / ANG2BOHR
    assert np.allclose(d.min(1), 1.48) and np.all(np.sort(d, 1)[:, 1] > 1.9)


def test_si353h196_and_bond_count():
    pos, z = silicon_cluster(WORKLOADS["si353h196"].r_cut_ang)
    nsi, nh = np.count_nonzero(z == 14), np.count_nonzero(z == 1)
    assert (nsi, nh) == (353, 196)
    si = pos[z == 14] / ANG2BOHR
    d = np.sqrt(((si[:, None] - si[None]) ** 2).sum(-1))
    bonds = np.count_nonzero(np.abs(d - 2.351) < 1e-2) // 2
    assert nh == 4 * nsi - 2 * bonds          # every dangling bond is capped once


def test_table1_occupation_and_dof():
    rows = np.loadtxt(GOLDEN)
    for n_si, n_h, h, d, npts, states, *_ in rows:
        z = np.array([14] * int(n_si) + [1] * int(n_h))
        nocc = n_occupied(z)
        assert nocc < states <= 1.3 * nocc
    last = rows[-1]
    assert abs(last[4] * last[5] / 7.8e12 - 1) < 0.01
    assert abs(last[5] / last[4] * 100 - 0.77) < 0.005


def test_rng_statistics_and_determinism():
    n = np.arange(400000)
    x = normal_entries(1, n)
    assert abs(x.mean()) < 0.01 and abs(x.std() - 1) < 0.01
    assert abs(np.mean(x ** 4) - 3) < 0.05
    assert np.array_equal(x[:1000], normal_entries(1, n[:1000]))
    assert not np.allclose(x[:1000], normal_entries(2, n[:1000]))
    blk = random_block_lex(3, 50, 7)
    sub = random_block_lex(3, 50, 7, points=[4, 9], cols=[6, 0])
    assert np.array_equal(sub, blk[[4, 9]][:, [6, 0]])
