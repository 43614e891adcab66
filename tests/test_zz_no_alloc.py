"""ea_c4_radial_noalloc, the entry point for callers that cannot allocate device
memory (a host whose device memory all belongs to its own pool, or a path where a
cudaMalloc, which may synchronise the device, is not allowed): its scratch is a
static array inside the library.  Its sums must equal those of ea_c4_radial, which
allocates its scratch, exactly (both are exact integers), call after call, although
every call reuses the same array.  Collected last, so that a stop at the first
failure has run every other test; it builds and loads the library itself, so it
also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def J():
    from paper_1411_5512_gb300 import build, job
    build.build()
    return job


def _call(lib, fn, j, t_w):
    from paper_1411_5512_gb300 import _lib
    nb = ctypes.c_int()
    assert lib.ea_c4_radial_bins(j.L, ctypes.byref(nb)) == 0
    sums = np.full((j.n_samples, nb.value), -7, dtype=np.int64)  # garbage to overwrite
    counts = np.full(nb.value, -7, dtype=np.int64)
    rc = getattr(lib, fn)(j.h, int(t_w), sums.ctypes.data_as(_lib.i64p),
                          counts.ctypes.data_as(_lib.i64p))
    return rc, sums, counts


@pytest.mark.parametrize("L,S,n", [(16, 3, 5), (128, 2, 2)])
def test_noalloc_matches_allocating_entry_point(J, L, S, n):
    j = J.EAJob(L, 0.5, 60 + L, S)
    j.set_schedule([0, n], [0])
    j.quench(0.7)
    j.sweep(n)
    lib = j.lib
    # two calls in a row on different snapshots, then the first again: the shared
    # scratch keeps the previous call's contents, which must not leak into the sums
    seen = []
    for t_w in (n, 0, n):
        rc, s_na, c_na = _call(lib, "ea_c4_radial_noalloc", j, t_w)
        assert rc == 0, lib.ea_last_error(j.h)
        rc, s_ref, c_ref = _call(lib, "ea_c4_radial", j, t_w)
        assert rc == 0, lib.ea_last_error(j.h)
        assert np.array_equal(c_na, c_ref)
        assert np.array_equal(s_na, s_ref), t_w
        seen.append(s_na)
    assert np.array_equal(seen[0], seen[2])
    assert not np.array_equal(seen[0], seen[1])  # the snapshots differ
    j.close()


def test_noalloc_rejects_sides_above_its_scratch(J):
    j = J.EAJob(130, 0.5, 3, 1)
    j.set_schedule([0], [0])
    j.quench(0.7)
    rc, _, _ = _call(j.lib, "ea_c4_radial_noalloc", j, 0)
    assert rc == -1  # EA_ERR_INVALID_ARG
    assert b"128" in j.lib.ea_last_error(j.h)
    j.close()
