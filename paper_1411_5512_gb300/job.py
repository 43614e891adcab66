"""Pythonic wrapper of one EA ageing job (a context of the C ABI).

Only argument marshalling happens here: every step of the simulation and of
the observables runs in the CUDA library.
"""
import ctypes

import numpy as np

from . import _lib

_torch_alloc_refs = None


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream or None
    return int(stream.cuda_stream)  # torch.cuda.Stream


def use_torch_allocator():
    """Route the library's device allocations through PyTorch's caching allocator."""
    global _torch_alloc_refs
    import torch

    lib = _lib.load()
    if _torch_alloc_refs is not None:
        return

    def _alloc(nbytes, stream, user):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), stream=stream or 0))
        except Exception:
            return None

    def _free(ptr, nbytes, stream, user):
        torch.cuda.caching_allocator_delete(int(ptr))

    a = _lib.ALLOC_FN(_alloc)
    f = _lib.FREE_FN(_free)
    _lib.check(lib.ea_set_allocator(a, f, None))
    _torch_alloc_refs = (a, f)


def use_cuda_allocator():
    """Back to the library's own cudaMalloc / cudaFree."""
    global _torch_alloc_refs
    lib = _lib.load()
    _lib.check(lib.ea_set_allocator(_lib.ALLOC_FN(), _lib.FREE_FN(), None))
    _torch_alloc_refs = None


def _host_ptr(buf, n_words):
    """Address of a host buffer of n_words 32-bit words (numpy array or torch tensor)."""
    if hasattr(buf, "data_ptr"):  # torch
        assert not buf.is_cuda and buf.element_size() == 4 and buf.numel() == n_words
        assert buf.is_contiguous()
        return buf.data_ptr()
    assert buf.dtype.itemsize == 4 and buf.size == n_words and buf.flags["C_CONTIGUOUS"]
    return buf.ctypes.data


def launch_count():
    """Kernel launches the library has issued in this process (a replayed graph
    counts the kernels it holds)."""
    return int(_lib.load().ea_launch_count())


def int_throughput(stream=None):
    """{"lop3", "imad", "philox"}: measured thread-ops/s (Philox: calls/s) of this GPU."""
    out = (ctypes.c_double * 3)()
    _lib.check(_lib.load().ea_int_throughput(_stream_handle(stream), out))
    return {"lop3": out[0], "imad": out[1], "philox": out[2]}


def debug_set_wait(polls, wait_for_nothing=False):
    """The bounded device waits: polls before giving up; wait_for_nothing (tests of
    the timeout path only) makes every wait run out."""
    _lib.check(_lib.load().ea_debug_set_wait(int(polls), 1 if wait_for_nothing else 0))


def device_status(stream=None):
    """Synchronise, read and clear the device status word (bit 0: a wait ran out)."""
    v = ctypes.c_uint32()
    rc = _lib.load().ea_device_status(_stream_handle(stream), ctypes.byref(v))
    if rc not in (_lib.EA_OK, _lib.EA_ERR_TIMEOUT):
        _lib.check(rc)
    return v.value


def geometry(L):
    out = (ctypes.c_int * 6)()
    _lib.check(_lib.load().ea_geometry(L, out))
    return tuple(out)


def thresholds(T, rule=0):
    thr = np.zeros(7, dtype=np.uint64)
    alw = np.zeros(7, dtype=np.uint8)
    _lib.check(_lib.load().ea_thresholds(float(T), int(rule),
                                         thr.ctypes.data_as(_lib.u64p),
                                         alw.ctypes.data_as(_lib.u8p)))
    return thr, alw


def footprint(L, n_samples, n_tw, n_t):
    b = ctypes.c_size_t()
    _lib.check(_lib.load().ea_footprint(L, n_samples, n_tw, n_t, ctypes.byref(b)))
    return b.value


class EAJob:
    """n_samples disorder samples x 2 replicas of an L^3 +-J EA lattice."""

    def __init__(self, L, p_neg, seed, n_samples, rng_group=1, stream=None, _handle=None,
                 exact_count=False, first_sample=0):
        """exact_count: exactly floor(p_neg 3N + 1/2) negative bonds per sample instead of
        independent bonds.  first_sample: this context holds the job's samples
        first_sample .. first_sample + n_samples - 1 (ea_create_samples_range)."""
        self.lib = _lib.load()
        self.L = int(L)
        self.n_samples = int(n_samples)
        self.first_sample = int(first_sample)
        self._stream = stream
        if _handle is not None:
            self.h = _handle
            return
        h = ctypes.c_void_p()
        if exact_count:
            assert self.first_sample == 0, "exact-count couplings cover whole jobs"
            _lib.check(self.lib.ea_create_samples_exact(
                ctypes.byref(h), self.L, float(p_neg), int(seed), self.n_samples, int(rng_group),
                _stream_handle(stream)))
        else:
            _lib.check(self.lib.ea_create_samples_range(
                ctypes.byref(h), self.L, float(p_neg), int(seed), self.first_sample,
                self.n_samples, int(rng_group), _stream_handle(stream)))
        self.h = h

    # -- lifecycle ---------------------------------------------------------------
    def set_schedule(self, t_w, t):
        tw = np.ascontiguousarray(np.array(list(t_w), dtype=np.uint64))
        tt = np.ascontiguousarray(np.array(list(t), dtype=np.uint64))
        _lib.check(self.lib.ea_set_schedule(self.h, tw.ctypes.data_as(_lib.u64p), len(tw),
                                            tt.ctypes.data_as(_lib.u64p), len(tt)), self.h)

    def quench(self, T, rule=0):
        _lib.check(self.lib.ea_quench(self.h, float(T), int(rule)), self.h)

    def sweep(self, n):
        _lib.check(self.lib.ea_sweep(self.h, int(n)), self.h)

    def set_row_range(self, y_lo, y_hi):
        """Sweeps update only the rows [y_lo, y_hi) (sides 64, 128; see domain.py)."""
        _lib.check(self.lib.ea_set_row_range(self.h, int(y_lo), int(y_hi)), self.h)

    def half_sweep(self):
        """The next half-step of the current sweep (h = 0, then h = 1)."""
        _lib.check(self.lib.ea_half_sweep(self.h), self.h)

    def get_rows(self, area, y, n_rows):
        """Rows y .. y + n_rows - 1 of spin area `area`, uint32 [S][n2][n_rows][n0]."""
        g = geometry(self.L)
        out = np.zeros((self.n_samples, g[5], n_rows, g[3]), dtype=np.uint32)
        _lib.check(self.lib.ea_get_rows(self.h, int(area), int(y), int(n_rows),
                                        out.ctypes.data_as(_lib.u32p)), self.h)
        return out

    def set_rows(self, area, y, words):
        arr = np.ascontiguousarray(words, dtype=np.uint32)
        _lib.check(self.lib.ea_set_rows(self.h, int(area), int(y), int(arr.shape[2]),
                                        arr.ctypes.data_as(_lib.u32p)), self.h)

    @property
    def time(self):
        t = ctypes.c_uint64()
        _lib.check(self.lib.ea_time(self.h, ctypes.byref(t)), self.h)
        return t.value

    def measure(self, t_w, t):
        S, R = self.n_samples, self.L // 2 + 1
        A = np.zeros((S, 2), dtype=np.int64)
        Q = np.zeros(S, dtype=np.int64)
        E = np.zeros((S, 2), dtype=np.int64)
        G = np.zeros((S, 3, R), dtype=np.int64)
        C4 = np.zeros(R, dtype=np.float64)
        sem = np.zeros(R, dtype=np.float64)
        obs = _lib.EaObs(A.ctypes.data_as(_lib.i64p), Q.ctypes.data_as(_lib.i64p),
                         E.ctypes.data_as(_lib.i64p), G.ctypes.data_as(_lib.i64p),
                         C4.ctypes.data_as(_lib.dblp), sem.ctypes.data_as(_lib.dblp),
                         0.0, 0.0, 0.0, 0)
        _lib.check(self.lib.ea_measure(self.h, int(t_w), int(t), ctypes.byref(obs)), self.h)
        return {"A": A, "Q": Q, "E": E, "G": G, "C4": C4, "C4_sem": sem, "C": obs.C,
                "q_mean": obs.q_mean, "xi1": obs.xi1, "r_cut": obs.r_cut}

    def c4_radial(self, t_w, noalloc=False):
        """Four-point sums over every displacement vector of the snapshot at t_w,
        binned by squared distance: {"sums": [S, n_bins], "counts": [n_bins],
        "r2", "r" (the occupied bins), "C4", "C4_sem" (the library's FP64 curve
        over the occupied bins)}.  noalloc: through ea_c4_radial_noalloc."""
        nb = ctypes.c_int()
        _lib.check(self.lib.ea_c4_radial_bins(int(self.L), ctypes.byref(nb)))
        sums = np.zeros((self.n_samples, nb.value), dtype=np.int64)
        counts = np.zeros(nb.value, dtype=np.int64)
        c4 = np.zeros(nb.value, dtype=np.float64)
        sem = np.zeros(nb.value, dtype=np.float64)
        fn = self.lib.ea_c4_radial_noalloc if noalloc else self.lib.ea_c4_radial
        _lib.check(fn(self.h, int(t_w), sums.ctypes.data_as(_lib.i64p),
                      counts.ctypes.data_as(_lib.i64p), c4.ctypes.data_as(_lib.dblp),
                      sem.ctypes.data_as(_lib.dblp)), self.h)
        occ = np.nonzero(counts)[0]
        return {"sums": sums, "counts": counts, "r2": occ, "r": np.sqrt(occ.astype(np.float64)),
                "C4": c4[occ], "C4_sem": sem[occ]}

    def spins(self, s, a):
        out = np.zeros((self.L,) * 3, dtype=np.int8)
        _lib.check(self.lib.ea_get_spins(self.h, int(s), int(a), out.ctypes.data_as(_lib.i8p)),
                   self.h)
        return out

    def all_spins(self, s):
        return np.stack([self.spins(s, 0), self.spins(s, 1)])

    def couplings(self, s):
        out = np.zeros((3,) + (self.L,) * 3, dtype=np.int8)
        _lib.check(self.lib.ea_get_couplings(self.h, int(s), out.ctypes.data_as(_lib.i8p)),
                   self.h)
        return out

    def set_spins(self, s, a, spins):
        arr = np.ascontiguousarray(spins, dtype=np.int8)
        assert arr.shape == (self.L,) * 3
        _lib.check(self.lib.ea_set_spins(self.h, int(s), int(a), arr.ctypes.data_as(_lib.i8p)),
                   self.h)

    def set_couplings(self, s, J):
        arr = np.ascontiguousarray(J, dtype=np.int8)
        assert arr.shape == (3,) + (self.L,) * 3
        _lib.check(self.lib.ea_set_couplings(self.h, int(s), arr.ctypes.data_as(_lib.i8p)),
                   self.h)

    def coupling_words(self, out=None):
        """All samples' couplings in the packed layout (uint32 words, see the C header);
        `out` may be a numpy array or a (pinned) torch tensor of that many 32-bit words."""
        n = ctypes.c_size_t()
        _lib.check(self.lib.ea_coupling_words(self.h, ctypes.byref(n)), self.h)
        if out is None:
            out = np.zeros(n.value, dtype=np.uint32)
        _lib.check(self.lib.ea_get_coupling_words(self.h, ctypes.c_void_p(_host_ptr(out, n.value))),
                   self.h)
        return out

    def set_coupling_words(self, words):
        """Replace the couplings by packed words from host memory (numpy array or
        torch tensor, 32-bit)."""
        n = ctypes.c_size_t()
        _lib.check(self.lib.ea_coupling_words(self.h, ctypes.byref(n)), self.h)
        _lib.check(self.lib.ea_set_coupling_words(self.h,
                                                  ctypes.c_void_p(_host_ptr(words, n.value))),
                   self.h)

    def set_time(self, t):
        _lib.check(self.lib.ea_set_time(self.h, int(t)), self.h)

    def thresholds(self):
        thr = np.zeros(7, dtype=np.uint64)
        alw = np.zeros(7, dtype=np.uint8)
        _lib.check(self.lib.ea_get_thresholds(self.h, thr.ctypes.data_as(_lib.u64p),
                                              alw.ctypes.data_as(_lib.u8p)), self.h)
        return thr, alw

    def checkpoint(self, path):
        _lib.check(self.lib.ea_checkpoint(self.h, str(path).encode()), self.h)

    @classmethod
    def restore(cls, path, stream=None):
        lib = _lib.load()
        h = ctypes.c_void_p()
        _lib.check(lib.ea_restore(ctypes.byref(h), str(path).encode(), _stream_handle(stream)))
        # read back shape from the file header: L and S are the 2nd and 3rd int32
        with open(path, "rb") as f:
            head = f.read(16)
        L, S = np.frombuffer(head[8:16], dtype=np.int32)
        return cls(int(L), 0.0, 0, int(S), stream=stream, _handle=h)

    def close(self):
        if getattr(self, "h", None) is not None and self.h:
            self.lib.ea_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class EABatch:
    """Many jobs swept together: one launch per half-step for all of them."""

    def __init__(self, stream=None):
        self.lib = _lib.load()
        h = ctypes.c_void_p()
        _lib.check(self.lib.ea_batch_create(ctypes.byref(h), _stream_handle(stream)))
        self.h = h
        self.jobs = []

    def add(self, job):
        _lib.check(self.lib.ea_batch_add(self.h, job.h), batch=self.h)
        self.jobs.append(job)

    def remove(self, job):
        _lib.check(self.lib.ea_batch_remove(self.h, job.h), batch=self.h)
        self.jobs.remove(job)

    def __len__(self):
        n = ctypes.c_int()
        _lib.check(self.lib.ea_batch_size(self.h, ctypes.byref(n)))
        return n.value

    def configure(self, cols_per_thread=0, graph_sweeps=0):
        _lib.check(self.lib.ea_batch_configure(self.h, int(cols_per_thread), int(graph_sweeps)),
                   batch=self.h)

    def config(self):
        a, b = ctypes.c_int(), ctypes.c_int()
        _lib.check(self.lib.ea_batch_get_config(self.h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def set_resident(self, max_side):
        """Metropolis members up to this side run sample-resident (0: never)."""
        _lib.check(self.lib.ea_batch_set_resident(self.h, int(max_side)), batch=self.h)

    def resident(self):
        v = ctypes.c_int()
        _lib.check(self.lib.ea_batch_get_resident(self.h, ctypes.byref(v)))
        return v.value

    def set_variant(self, variant):
        """Side-128 Metropolis members: 1 the staged kernel, 0 the tile kernel."""
        _lib.check(self.lib.ea_batch_set_variant(self.h, int(variant)), batch=self.h)

    def variant(self):
        v = ctypes.c_int()
        _lib.check(self.lib.ea_batch_get_variant(self.h, ctypes.byref(v)))
        return v.value

    def set_streams(self, streams):
        """Members on one kernel are split into this many groups of whole jobs, each
        swept on a stream of its own (1 .. 5; 1: one launch per half-step for all)."""
        _lib.check(self.lib.ea_batch_set_streams(self.h, int(streams)), batch=self.h)

    def streams(self):
        v = ctypes.c_int()
        _lib.check(self.lib.ea_batch_get_streams(self.h, ctypes.byref(v)))
        return v.value

    def autotune(self, trial_sweeps=8):
        _lib.check(self.lib.ea_batch_autotune(self.h, int(trial_sweeps)), batch=self.h)
        return self.config()

    def sweep(self, n):
        _lib.check(self.lib.ea_batch_sweep(self.h, int(n)), batch=self.h)

    def profile(self, sweeps=4):
        """{words, philox_calls, rare_calls, flips} over `sweeps` counted sweeps (the
        members' state is put back afterwards).  philox_calls counts every call;
        rare_calls the extension and continuation calls of the rare path among them."""
        out = np.zeros(4, dtype=np.uint64)
        _lib.check(self.lib.ea_batch_profile(self.h, int(sweeps), out.ctypes.data_as(_lib.u64p)),
                   batch=self.h)
        return {"words": int(out[0]), "philox_calls": int(out[1]),
                "rare_calls": int(out[2]), "flips": int(out[3])}

    def close(self):
        if getattr(self, "h", None) is not None and self.h:
            self.lib.ea_batch_destroy(self.h)
            self.h = None
            self.jobs = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class EAServer:
    """Continuous batching of ageing jobs (admission by device footprint)."""

    def __init__(self, budget_bytes, max_running=64, chunk_sweeps=256, stream=None):
        self.lib = _lib.load()
        h = ctypes.c_void_p()
        _lib.check(self.lib.ea_server_create(ctypes.byref(h), int(budget_bytes), int(max_running),
                                             int(chunk_sweeps), _stream_handle(stream)))
        self.h = h
        self._keep = {}

    def submit(self, L, p_neg, seed, n_samples, T, sweeps, t_w=(), t=(), rule=0, rng_group=1):
        tw = np.ascontiguousarray(np.array(list(t_w), dtype=np.uint64))
        tt = np.ascontiguousarray(np.array(list(t), dtype=np.uint64))
        spec = _lib.EaJobSpec(int(L), float(p_neg), int(seed), int(n_samples), int(rng_group),
                              float(T), int(rule), int(sweeps), tw.ctypes.data_as(_lib.u64p),
                              len(tw), tt.ctypes.data_as(_lib.u64p), len(tt))
        jid = ctypes.c_int64()
        _lib.check(self.lib.ea_server_submit(self.h, ctypes.byref(spec), ctypes.byref(jid)),
                   server=self.h)
        self._keep[jid.value] = (int(L), int(n_samples))
        return jid.value

    def configure(self, cols_per_thread=4, graph_sweeps=16):
        _lib.check(self.lib.ea_server_configure(self.h, int(cols_per_thread), int(graph_sweeps)),
                   server=self.h)

    def step(self):
        n = ctypes.c_int()
        _lib.check(self.lib.ea_server_step(self.h, ctypes.byref(n)), server=self.h)
        return n.value

    def state(self, job_id):
        st = ctypes.c_int()
        t = ctypes.c_uint64()
        _lib.check(self.lib.ea_server_job_state(self.h, int(job_id), ctypes.byref(st),
                                                ctypes.byref(t)), server=self.h)
        return st.value, t.value

    def job(self, job_id):
        """The job's context as an EAJob view (owned by the server)."""
        h = ctypes.c_void_p()
        _lib.check(self.lib.ea_server_job(self.h, int(job_id), ctypes.byref(h)), server=self.h)
        L, S = self._keep[int(job_id)]
        view = EAJob(L, 0.0, 0, S, _handle=h)
        view.close = lambda: None  # the server owns it
        return view

    def release(self, job_id):
        _lib.check(self.lib.ea_server_release(self.h, int(job_id)), server=self.h)
        self._keep.pop(int(job_id), None)

    def cancel(self, job_id):
        _lib.check(self.lib.ea_server_cancel(self.h, int(job_id)), server=self.h)
        self._keep.pop(int(job_id), None)

    def stats(self):
        st = _lib.EaServerStats()
        _lib.check(self.lib.ea_server_get_stats(self.h, ctypes.byref(st)))
        return {"queued": st.queued, "running": st.running, "done": st.done,
                "bytes_in_use": st.bytes_in_use, "flips": st.flips, "steps": st.steps}

    def close(self):
        if getattr(self, "h", None) is not None and self.h:
            self.lib.ea_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
