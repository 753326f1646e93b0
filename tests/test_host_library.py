"""Host-side checks of the C-ABI library (no GPU): every symbol declared in
include/*.h is exported, the Hilbert brick order, and the grid tables against the
oracle's grid."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def kscf():
    from paper_2303_00790_gb300.build import build
    build()
    from paper_2303_00790_gb300 import kscf as mod
    return mod


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(kscf_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_exports_every_declared_symbol(kscf):
    names = declared_functions()
    assert len(names) >= 18
    lib = ctypes.CDLL(kscf.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(kscf.EXPORTED) >= names


def test_hilbert_index_is_a_continuous_bijection(kscf):
    bits = 3
    n = 1 << bits
    idx = {}
    for x in range(n):
        for y in range(n):
            for z in range(n):
                idx[kscf.kscf_hilbert_index3(x, y, z, bits)] = (x, y, z)
    assert sorted(idx) == list(range(n ** 3))
    for t in range(n ** 3 - 1):
        a, b = np.array(idx[t]), np.array(idx[t + 1])
        assert np.abs(a - b).sum() == 1
    assert idx[0] == (0, 0, 0)


@pytest.mark.parametrize("brick", [8, 16])
def test_sphere_grid_tables_match_oracle(kscf, brick):
    from oracle.grid import sphere_grid
    c, R, h = (0.3, -0.1, 0.2), 9.3, 0.7
    g = kscf.kscf_build_grid(c, R, h, brick)
    og = sphere_grid(c, R, h)
    info = g.info
    assert info["n_points"] == og.n
    lex, ijk = g.slots()
    live = lex >= 0
    assert live.sum() == og.n
    assert np.array_equal(np.sort(lex[live]), np.arange(og.n))
    assert np.array_equal(ijk[live], og.ijk[lex[live]])              # same point in each slot
    assert info["n_slots"] == info["n_bricks"] * brick ** 3
    # slots inside a brick are x-fastest; bricks are visited along the Hilbert curve
    b3 = brick ** 3
    bc = (ijk[::b3] - np.array(info["lo"])) // brick
    bits = int(np.ceil(np.log2(max(1, (np.array(info["extent"]) + brick - 1).max() // brick))))
    keys = [kscf.kscf_hilbert_index3(int(x), int(y), int(z), bits) for x, y, z in bc]
    assert all(k1 < k2 for k1, k2 in zip(keys, keys[1:]))
    first = ijk[:b3] - ijk[0]
    assert tuple(first[1]) == (1, 0, 0) and tuple(first[brick]) == (0, 1, 0)
    assert tuple(first[brick * brick]) == (0, 0, 1)


def test_box_grid_and_errors(kscf):
    g = kscf.kscf_build_grid_box(9, 10, 11, 0.5, 8)
    assert g.info["n_points"] == 990 and g.info["n_bricks"] == 8
    lex, ijk = g.slots()
    assert (lex >= 0).sum() == 990
    with pytest.raises(kscf.KscfError) as e:
        kscf.kscf_build_grid((0, 0, 0), 5.0, 0.7, 12)
    assert e.value.code == kscf.KSCF_ERR_INVALID
    with pytest.raises(kscf.KscfError):
        kscf.kscf_build_grid((0, 0, 0), -1.0, 0.7, 8)


def test_workload_grid_sizes(kscf):
    from workloads import WORKLOADS
    w = WORKLOADS["si35h36"]
    pos, z = w.atoms()
    g = kscf.kscf_build_grid(pos[0], w.radius, w.h, 8)
    assert g.info["n_points"] == 45025
