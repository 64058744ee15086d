"""CPU-side checks of the C ABI: the library builds, loads, exports every
function include/hacc.h declares, and its host-only entry points behave."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def _declared():
    names = []
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"\b(hacc_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1410_2805_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("hacc_bin", "hacc_sr_force", "hacc_subcycle", "hacc_step"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_default_split_matches_oracle_fit():
    import paper_1410_2805_gb300 as hacc
    from oracle import split
    s = hacc.default_split()
    o = split.default_split()
    assert s.r_cut == np.float32(o["r_cut"])
    assert s.eps == np.float32(o["eps"])
    # two independent FP64 fits (Householder QR here, numpy's SVD there)
    assert np.allclose(s.poly, o["poly"], rtol=1e-9, atol=0)


def test_mesh_cells_rule():
    import paper_1410_2805_gb300 as hacc
    rc = hacc.default_split().r_cut
    assert hacc.mesh_cells(32.0, rc) == 10
    assert hacc.mesh_cells(256.0, rc) == 82
    assert hacc.mesh_cells(512.0, rc) == 164
    assert hacc.mesh_cells(8.0, rc) == -1            # fewer than 3 cells
    assert hacc.mesh_cells(3.0 * rc, rc) == -1        # width would equal r_cut: one fewer


def test_ml_mesh_cells_rule():
    import paper_1410_2805_gb300 as hacc
    rc = hacc.default_split().r_cut
    # cells at least 1.05 r_cut wide: floor(128 / (1.05 rc)) = 39 < 41
    assert hacc.mesh_cells(128.0, rc) == 41
    assert hacc.ml_mesh_cells(128.0, rc, 0.05) == 39
    assert hacc.ml_mesh_cells(128.0, rc, 0.0) == 41
    # the slack of 20 / 6 already covers 5 %: unchanged
    assert hacc.ml_mesh_cells(20.0, rc, 0.05) == hacc.mesh_cells(20.0, rc) == 6
    # never below 3 cells: a 3-cell box keeps 3
    assert hacc.ml_mesh_cells(10.0, rc, 0.5) == 3
    assert hacc.ml_mesh_cells(8.0, rc, 0.05) == -1


def test_batch_scratch_bytes_is_host_arithmetic():
    # the serving admission's footprint query runs without a device
    import paper_1410_2805_gb300 as hacc
    from paper_1410_2805_gb300 import build
    build.build()
    sp = hacc.default_split()
    one = [hacc.BatchBox(L=18.0, offset=0, n=5000, dt=0.01)]
    two = one + [hacc.BatchBox(L=24.0, offset=5000, n=12000, dt=0.01)]
    s1, s2 = hacc.batch_scratch_bytes(sp, one), hacc.batch_scratch_bytes(sp, two)
    assert 5000 * 64 < s1 < s2
    # per particle about 83 bytes plus 32 per cell at large sizes
    big = hacc.batch_scratch_bytes(sp, [hacc.BatchBox(L=256.0, offset=0, n=256 ** 3, dt=0.01)])
    assert 75 * 256 ** 3 < big < 95 * 256 ** 3
    assert hacc.batch_scratch_bytes(sp, []) == 0
    assert hacc.batch_scratch_bytes(sp, [hacc.BatchBox(L=18.0, offset=0, n=0, dt=0.01)]) == 0
    assert hacc.batch_scratch_bytes(sp, [hacc.BatchBox(L=5.0, offset=0, n=10, dt=0.01)]) == 0   # < 3 cells
