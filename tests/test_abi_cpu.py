"""CPU checks of the C ABI: the library builds, loads, exports every symbol the
header declares, and its host-only helpers agree with the oracle.  No call here
touches a GPU."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import oracle as ora

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ea_ageing.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1411_5512_gb300 import build, _lib
    build.build()
    return _lib.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\**\s*(ea_[a-z_0-9]+)\s*\(", text, re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["ea_create_samples", "ea_set_schedule", "ea_quench", "ea_sweep", "ea_measure",
              "ea_get_spins", "ea_get_couplings", "ea_get_thresholds", "ea_checkpoint",
              "ea_restore", "ea_destroy", "ea_last_error", "ea_geometry", "ea_thresholds"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1411_5512_gb300 import _lib
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, name


def test_geometry_matches_oracle(lib):
    from paper_1411_5512_gb300 import job
    for L in [2, 4, 6, 8, 10, 12, 16, 20, 24, 32, 48, 64, 96, 128, 256, 1024]:
        assert job.geometry(L) == ora.geometry(L)
    out = (ctypes.c_int * 6)()
    for L in [0, 1, 3, 7, 1025, 2048, -4]:
        assert lib.ea_geometry(L, out) == -1


def test_c4_radial_bins(lib):
    nb = ctypes.c_int()
    for L in [2, 4, 6, 16, 128, 512]:
        assert lib.ea_c4_radial_bins(L, ctypes.byref(nb)) == 0
        assert nb.value == 3 * (L // 2) ** 2 + 1
        if L <= 16:  # the oracle's binning has as many bins
            assert nb.value == len(ora.c4_radial_sums(np.zeros((L, L, L), dtype=np.int64))[1])
    for L in [0, 3, 514, 1024]:
        assert lib.ea_c4_radial_bins(L, ctypes.byref(nb)) == -1


@pytest.mark.parametrize("rule", [0, 1])
def test_thresholds_match_oracle(lib, rule):
    from paper_1411_5512_gb300 import job
    for T in [0.0, 0.3, 0.5, 0.6, 0.7, 0.8, 1.0, 1.1, 2.5, 4.0 / math.log(2.0), 1e6,
              float("inf")]:
        t1, a1 = job.thresholds(T, rule)
        t2, a2 = ora.thresholds(T, rule)
        assert np.array_equal(t1, t2) and np.array_equal(a1, a2), T


def test_invalid_arguments_need_no_gpu(lib):
    h = ctypes.c_void_p()
    # odd L, L too small, p outside [0, 1], no samples, bad share group
    for args in [(15, 0.5, 1, 1, 1), (0, 0.5, 1, 1, 1), (16, 1.5, 1, 1, 1),
                 (16, -0.1, 1, 1, 1), (16, 0.5, 1, 0, 1), (16, 0.5, 1, 1, 0),
                 (16, float("nan"), 1, 1, 1)]:
        assert lib.ea_create_samples(ctypes.byref(h), *args, None) == -1
    thr = np.zeros(7, dtype=np.uint64)
    alw = np.zeros(7, dtype=np.uint8)
    from paper_1411_5512_gb300 import _lib
    assert lib.ea_thresholds(-1.0, 0, thr.ctypes.data_as(_lib.u64p),
                             alw.ctypes.data_as(_lib.u8p)) == -1
    assert lib.ea_thresholds(1.0, 5, thr.ctypes.data_as(_lib.u64p),
                             alw.ctypes.data_as(_lib.u8p)) == -1
    assert lib.ea_destroy(None) == 0
    assert lib.ea_last_error(None) == b""
    assert lib.ea_status_string(-3) == b"EA_ERR_NO_SNAPSHOT"


def test_footprint(lib):
    from paper_1411_5512_gb300 import job
    # L = 128: 65536 words per sample; 2 spin areas + 3 coupling planes = 20 B/word-site
    b = job.footprint(128, 16, 0, 0)
    assert b == 16 * 65536 * 4 * 5
    assert job.footprint(128, 16, 4, 4) > b


def test_geo_table_matches_oracle(lib):
    import numpy as np
    from paper_1411_5512_gb300 import _lib
    for T in (0.5, 0.6, 0.7, 0.8, 1.0, 3.0):
        for dE in (4, 8, 12):
            p = math.exp(-dE / T)
            C = np.zeros(33, dtype=np.uint64)
            assert lib.ea_geo_table(p, C.ctypes.data_as(_lib.u64p)) == 0
            assert np.array_equal(C, ora.geo_table(p)), (T, dE)
    C = np.zeros(33, dtype=np.uint64)
    for bad in (0.0, 1.0, -1.0):
        assert lib.ea_geo_table(bad, C.ctypes.data_as(_lib.u64p)) == -1
