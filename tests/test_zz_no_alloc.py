"""ea_c4_radial_noalloc, the entry point for callers that cannot allocate device
memory (a host whose device memory all belongs to its own pool, or a path where a
cudaMalloc, which may synchronise the device, is not allowed): its scratch is a
static array inside the library.  Its sums must equal those of ea_c4_radial, which
allocates its scratch, exactly (both are exact integers), call after call, although
every call reuses the same array; and it must keep working while every allocation
is refused, where ea_c4_radial reports EA_ERR_OOM.  Collected last, so that a stop
at the first failure has run every other test; it builds and loads the library
itself, so it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

EA_ERR_OOM = -2


@pytest.fixture(scope="module")
def J():
    from paper_1411_5512_gb300 import build, job
    build.build()
    return job


class RefusingAllocator:
    """Installed as the library's allocator: refuses every request and records
    every call; the library's own cudaMalloc / cudaFree come back on exit."""

    def __init__(self):
        from paper_1411_5512_gb300 import _lib
        self._lib = _lib
        self.calls = []

        def _alloc(nbytes, stream, user):
            self.calls.append(("alloc", int(nbytes)))
            return None

        def _free(ptr, nbytes, stream, user):
            self.calls.append(("free", int(nbytes)))

        self.a = _lib.ALLOC_FN(_alloc)
        self.f = _lib.FREE_FN(_free)

    def __enter__(self):
        self._lib.check(self._lib.load().ea_set_allocator(self.a, self.f, None))
        return self

    def __exit__(self, *exc):
        self._lib.check(self._lib.load().ea_set_allocator(self._lib.ALLOC_FN(),
                                                          self._lib.FREE_FN(), None))


def _call(lib, fn, j, t_w):
    from paper_1411_5512_gb300 import _lib
    nb = ctypes.c_int()
    assert lib.ea_c4_radial_bins(j.L, ctypes.byref(nb)) == 0
    sums = np.full((j.n_samples, nb.value), -7, dtype=np.int64)  # garbage to overwrite
    counts = np.full(nb.value, -7, dtype=np.int64)
    c4 = np.full(nb.value, -7.0)
    sem = np.full(nb.value, -7.0)
    rc = getattr(lib, fn)(j.h, int(t_w), sums.ctypes.data_as(_lib.i64p),
                          counts.ctypes.data_as(_lib.i64p), c4.ctypes.data_as(_lib.dblp),
                          sem.ctypes.data_as(_lib.dblp))
    return rc, sums, counts, c4, sem


def _same_curve(a, b):
    return bool(np.all((a == b) | (np.isnan(a) & np.isnan(b))))


# side 16 and 128 take the radix-2 transform, 24 and 96 the direct DFT
@pytest.mark.parametrize("L,S,n", [(16, 3, 5), (24, 3, 5), (96, 2, 2), (128, 2, 2)])
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
        rc, s_na, c_na, c4_na, sem_na = _call(lib, "ea_c4_radial_noalloc", j, t_w)
        assert rc == 0, lib.ea_last_error(j.h)
        rc, s_ref, c_ref, c4_ref, sem_ref = _call(lib, "ea_c4_radial", j, t_w)
        assert rc == 0, lib.ea_last_error(j.h)
        assert np.array_equal(c_na, c_ref)
        assert np.array_equal(s_na, s_ref), t_w
        assert _same_curve(c4_na, c4_ref) and _same_curve(sem_na, sem_ref), t_w
        seen.append(s_na)
    assert np.array_equal(seen[0], seen[2])
    assert not np.array_equal(seen[0], seen[1])  # the snapshots differ
    # with every allocation refused: the entry point without allocation asks for
    # nothing and still gives the same sums; the allocating one reports EA_ERR_OOM
    with RefusingAllocator() as ra:
        rc, s_na, c_na, c4_na, _ = _call(lib, "ea_c4_radial_noalloc", j, n)
        assert rc == 0, lib.ea_last_error(j.h)
        assert ra.calls == []
        assert np.array_equal(s_na, seen[0]) and np.array_equal(c_na, c_ref)
        rc, *_ = _call(lib, "ea_c4_radial", j, n)
        assert rc == EA_ERR_OOM
        assert ra.calls and all(kind == "alloc" for kind, _ in ra.calls)
    j.close()


def test_noalloc_matches_the_oracle(J):
    """Directly against the oracle's brute force over every displacement vector, on the
    oracle's own spins (side 16, two samples)."""
    import oracle as ora
    L, S, n, seed = 16, 2, 4, 71
    j = J.EAJob(L, 0.5, seed, S)
    j.set_schedule([n], [0])
    j.quench(0.7)
    j.sweep(n)
    rc, sums, counts, _, _ = _call(j.lib, "ea_c4_radial_noalloc", j, n)
    assert rc == 0, j.lib.ea_last_error(j.h)
    ref = ora.run_job(L, 0.5, seed, S, 0.7, 0, [], [], n, keep_spins=True)
    for s in range(S):
        want, want_counts = ora.c4_radial_sums(ora.c4_full_sums(ref["spins"][s]))
        assert np.array_equal(counts, want_counts)
        assert np.array_equal(sums[s], want), s
    j.close()


def test_noalloc_rejects_sides_above_its_scratch(J):
    j = J.EAJob(130, 0.5, 3, 1)
    j.set_schedule([0], [0])
    j.quench(0.7)
    rc, *_ = _call(j.lib, "ea_c4_radial_noalloc", j, 0)
    assert rc == -1  # EA_ERR_INVALID_ARG
    assert b"128" in j.lib.ea_last_error(j.h)
    j.close()
