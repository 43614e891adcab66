"""ctypes binding of the C ABI in include/ea_ageing.h (argument marshalling only).

Every function of the header is exposed under its own name with its C
signature.  Loading fails loudly when the compiled library is missing: there is
no CPU fallback.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libea_gb300.so")

EA_OK = 0
EA_ERR_INVALID_ARG = -1
EA_ERR_OOM = -2
EA_ERR_NO_SNAPSHOT = -3
EA_ERR_STATE = -4
EA_ERR_TIMEOUT = -5
EA_ERR_CUDA = -6
EA_ERR_IO = -7

EA_RULE_METROPOLIS = 0
EA_RULE_HEATBATH = 1

i64p = ctypes.POINTER(ctypes.c_int64)
u64p = ctypes.POINTER(ctypes.c_uint64)
u8p = ctypes.POINTER(ctypes.c_uint8)
i8p = ctypes.POINTER(ctypes.c_int8)
u32p = ctypes.POINTER(ctypes.c_uint32)
dblp = ctypes.POINTER(ctypes.c_double)
intp = ctypes.POINTER(ctypes.c_int)
vp = ctypes.c_void_p


class EaObs(ctypes.Structure):
    _fields_ = [("A", i64p), ("Q", i64p), ("E", i64p), ("G", i64p),
                ("C4", dblp), ("C4_sem", dblp),
                ("C", ctypes.c_double), ("q_mean", ctypes.c_double),
                ("xi1", ctypes.c_double), ("r_cut", ctypes.c_int)]


class EaJobSpec(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("p_neg", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("n_samples", ctypes.c_int), ("rng_group_G", ctypes.c_int),
                ("T", ctypes.c_double), ("rule", ctypes.c_int), ("sweeps", ctypes.c_uint64),
                ("t_w", u64p), ("n_tw", ctypes.c_int), ("t", u64p), ("n_t", ctypes.c_int)]


class EaServerStats(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_int), ("running", ctypes.c_int), ("done", ctypes.c_int),
                ("bytes_in_use", ctypes.c_size_t), ("flips", ctypes.c_uint64),
                ("steps", ctypes.c_uint64)]


EA_JOB_QUEUED = 0
EA_JOB_RUNNING = 1
EA_JOB_DONE = 2

ALLOC_FN = ctypes.CFUNCTYPE(vp, ctypes.c_size_t, vp, vp)
FREE_FN = ctypes.CFUNCTYPE(None, vp, ctypes.c_size_t, vp, vp)

# name -> (restype, argtypes), in header order
SIGNATURES = {
    "ea_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "ea_geometry": (ctypes.c_int, [ctypes.c_int, intp]),
    "ea_thresholds": (ctypes.c_int, [ctypes.c_double, ctypes.c_int, u64p, u8p]),
    "ea_geo_table": (ctypes.c_int, [ctypes.c_double, u64p]),
    "ea_footprint": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_size_t)]),
    "ea_set_allocator": (ctypes.c_int, [ALLOC_FN, FREE_FN, vp]),
    "ea_int_throughput": (ctypes.c_int, [vp, dblp]),
    "ea_debug_set_wait": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_int]),
    "ea_device_status": (ctypes.c_int, [vp, u32p]),
    "ea_create_samples": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_double,
                                         ctypes.c_uint64, ctypes.c_int, ctypes.c_int, vp]),
    "ea_create_samples_exact": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_double,
                                               ctypes.c_uint64, ctypes.c_int, ctypes.c_int, vp]),
    "ea_create_samples_range": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_double,
                                               ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_int, vp]),
    "ea_set_schedule": (ctypes.c_int, [vp, u64p, ctypes.c_int, u64p, ctypes.c_int]),
    "ea_quench": (ctypes.c_int, [vp, ctypes.c_double, ctypes.c_int]),
    "ea_sweep": (ctypes.c_int, [vp, ctypes.c_uint64]),
    "ea_set_row_range": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int]),
    "ea_half_sweep": (ctypes.c_int, [vp]),
    "ea_get_rows": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, u32p]),
    "ea_set_rows": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, u32p]),
    "ea_time": (ctypes.c_int, [vp, u64p]),
    "ea_measure": (ctypes.c_int, [vp, ctypes.c_uint64, ctypes.c_uint64,
                                  ctypes.POINTER(EaObs)]),
    "ea_c4_radial": (ctypes.c_int, [vp, ctypes.c_uint64, i64p, i64p, dblp, dblp]),
    "ea_c4_radial_noalloc": (ctypes.c_int, [vp, ctypes.c_uint64, i64p, i64p, dblp, dblp]),
    "ea_c4_radial_bins": (ctypes.c_int, [ctypes.c_int, intp]),
    "ea_get_spins": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, i8p]),
    "ea_get_couplings": (ctypes.c_int, [vp, ctypes.c_int, i8p]),
    "ea_set_spins": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, i8p]),
    "ea_set_couplings": (ctypes.c_int, [vp, ctypes.c_int, i8p]),
    "ea_set_time": (ctypes.c_int, [vp, ctypes.c_uint64]),
    "ea_coupling_words": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_size_t)]),
    "ea_get_coupling_words": (ctypes.c_int, [vp, vp]),
    "ea_set_coupling_words": (ctypes.c_int, [vp, vp]),
    "ea_get_thresholds": (ctypes.c_int, [vp, u64p, u8p]),
    "ea_checkpoint": (ctypes.c_int, [vp, ctypes.c_char_p]),
    "ea_restore": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_char_p, vp]),
    "ea_destroy": (ctypes.c_int, [vp]),
    "ea_last_error": (ctypes.c_char_p, [vp]),
    "ea_batch_create": (ctypes.c_int, [ctypes.POINTER(vp), vp]),
    "ea_batch_add": (ctypes.c_int, [vp, vp]),
    "ea_batch_remove": (ctypes.c_int, [vp, vp]),
    "ea_batch_size": (ctypes.c_int, [vp, intp]),
    "ea_batch_configure": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int]),
    "ea_batch_get_config": (ctypes.c_int, [vp, intp, intp]),
    "ea_batch_set_resident": (ctypes.c_int, [vp, ctypes.c_int]),
    "ea_batch_get_resident": (ctypes.c_int, [vp, intp]),
    "ea_batch_set_variant": (ctypes.c_int, [vp, ctypes.c_int]),
    "ea_batch_get_variant": (ctypes.c_int, [vp, intp]),
    "ea_batch_set_streams": (ctypes.c_int, [vp, ctypes.c_int]),
    "ea_batch_get_streams": (ctypes.c_int, [vp, intp]),
    "ea_batch_autotune": (ctypes.c_int, [vp, ctypes.c_int]),
    "ea_batch_profile": (ctypes.c_int, [vp, ctypes.c_int, u64p]),
    "ea_batch_sweep": (ctypes.c_int, [vp, ctypes.c_uint64]),
    "ea_batch_destroy": (ctypes.c_int, [vp]),
    "ea_batch_last_error": (ctypes.c_char_p, [vp]),
    "ea_server_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_size_t, ctypes.c_int,
                                        ctypes.c_uint64, vp]),
    "ea_server_submit": (ctypes.c_int, [vp, ctypes.POINTER(EaJobSpec),
                                        ctypes.POINTER(ctypes.c_int64)]),
    "ea_server_step": (ctypes.c_int, [vp, intp]),
    "ea_server_configure": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int]),
    "ea_server_job_state": (ctypes.c_int, [vp, ctypes.c_int64, intp, u64p]),
    "ea_server_job": (ctypes.c_int, [vp, ctypes.c_int64, ctypes.POINTER(vp)]),
    "ea_server_release": (ctypes.c_int, [vp, ctypes.c_int64]),
    "ea_server_cancel": (ctypes.c_int, [vp, ctypes.c_int64]),
    "ea_server_get_stats": (ctypes.c_int, [vp, ctypes.POINTER(EaServerStats)]),
    "ea_server_destroy": (ctypes.c_int, [vp]),
    "ea_launch_count": (ctypes.c_uint64, []),
    "ea_server_last_error": (ctypes.c_char_p, [vp]),
}

_lib = None


def load(path=LIB_PATH):
    """Load the compiled library; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            "libea_gb300.so is not built (%s); run __graft_entry__.build() or "
            "python -m paper_1411_5512_gb300.build" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class EAError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        name = load().ea_status_string(status).decode()
        super().__init__("%s%s" % (name, (": " + msg) if msg else ""))


def check(status, ctx=None, batch=None, server=None):
    if status != EA_OK:
        msg = ""
        if ctx is not None:
            msg = (load().ea_last_error(ctx) or b"").decode()
        if batch is not None:
            msg = (load().ea_batch_last_error(batch) or b"").decode()
        if server is not None:
            msg = (load().ea_server_last_error(server) or b"").decode()
        raise EAError(status, msg)
    return status
