"""ctypes binding of libsuperdc.so (argument marshalling only).

Every numeric step runs in the CUDA library; this module passes raw device
pointers (``tensor.data_ptr()``) and the current CUDA stream.  There is no
CPU fallback: if the library cannot be built or loaded, or no CUDA device is
present, calls raise.
"""
import ctypes
import os

from . import build as _build

c_double, c_int32, c_int64, c_void_p = ctypes.c_double, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p

STATUS = {0: "SUPERDC_OK", 1: "SUPERDC_ERR_ARG", 2: "SUPERDC_ERR_CUDA", 3: "SUPERDC_ERR_OOM",
          4: "SUPERDC_ERR_NONFINITE", 5: "SUPERDC_ERR_NOCONV", 6: "SUPERDC_ERR_STATE"}
DEV_NONFINITE, DEV_NOCONV, DEV_INDEX = 1, 2, 4


class SuperDCError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        super().__init__("%s%s" % (STATUS.get(code, "status %d" % code), (" in " + where) if where else ""))


class Opts(ctypes.Structure):
    _fields_ = [("tau", c_double), ("stop_c", c_double), ("max_iter", c_int32),
                ("tile_roots", c_int32), ("batching", c_int32), ("sched", c_int32), ("tape", c_int32),
                ("fmm_min_m", c_int32), ("shifted", c_int32), ("balanced", c_int32)]


class Tree(ctypes.Structure):
    _fields_ = [("n", c_int64), ("nnodes", c_int32), ("lchild", c_void_p), ("rchild", c_void_p),
                ("leaf_size", c_void_p), ("rank", c_int32)]


class MatrixEntries(ctypes.Structure):
    _fields_ = [("kind", c_int32), ("A", c_void_p), ("lda", c_int64), ("x", c_void_p), ("param", c_double)]


class Rank1Out(ctypes.Structure):
    _fields_ = [(n, c_void_p) for n in ("lam", "dk", "zk", "eta", "vhat", "bnorm", "org", "src", "perm",
                                         "giv_ab", "giv_cs", "mk", "ngiv", "sweeps", "status", "fmm")]


_lib = None


def lib():
    """Load (building in-tree if needed) the CUDA library; with the
    environment variable SUPERDC_CHECKED=1 the checked build (index guards
    latch SUPERDC_DEV_INDEX, reported as SUPERDC_ERR_CUDA)."""
    global _lib
    if _lib is None:
        path = _build.build(check=os.environ.get("SUPERDC_CHECKED", "0") == "1")
        if not os.path.exists(path):
            raise RuntimeError("libsuperdc.so missing at %s" % path)
        L = ctypes.CDLL(path)
        L.superdc_opts_default.argtypes = [ctypes.POINTER(Opts)]
        L.superdc_opts_default.restype = c_int32
        L.superdc_debug_alloc_limit.argtypes = [c_int64]
        L.superdc_debug_alloc_limit.restype = c_int32
        L.superdc_status_string.argtypes = [c_int32]
        L.superdc_status_string.restype = ctypes.c_char_p
        L.superdc_secular_batched.argtypes = [c_int64, c_void_p, c_int64, c_void_p, c_void_p, c_double,
                                              ctypes.POINTER(Opts), ctypes.POINTER(Rank1Out), c_void_p]
        L.superdc_secular_batched.restype = c_int32
        L.superdc_secular_batched_host.argtypes = [c_int64, c_void_p, c_int64, c_void_p, c_void_p, c_double,
                                                   ctypes.POINTER(Opts), ctypes.POINTER(Rank1Out), c_void_p]
        L.superdc_secular_batched_host.restype = c_int32
        L.superdc_build_hss.argtypes = [ctypes.POINTER(Tree), c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                        ctypes.POINTER(c_void_p)]
        L.superdc_build_hss.restype = c_int32
        L.superdc_build_hss_hermitian.argtypes = [ctypes.POINTER(Tree), c_void_p, c_void_p, c_void_p, c_void_p,
                                                  c_void_p, ctypes.POINTER(c_void_p)]
        L.superdc_build_hss_hermitian.restype = c_int32
        L.superdc_hss_get.argtypes = [c_void_p, ctypes.c_char_p, c_void_p]
        L.superdc_hss_get.restype = c_int32
        L.superdc_build_hss_compress.argtypes = [c_int64, c_int32, c_int32, ctypes.POINTER(MatrixEntries), c_void_p,
                                                 c_int32, c_void_p, ctypes.POINTER(c_void_p),
                                                 ctypes.POINTER(c_double)]
        L.superdc_build_hss_compress.restype = c_int32
        L.superdc_hss_free.argtypes = [c_void_p]
        L.superdc_hss_free.restype = None
        L.superdc_eig.argtypes = [c_void_p, ctypes.POINTER(Opts), c_void_p, c_void_p, ctypes.POINTER(c_void_p)]
        L.superdc_eig.restype = c_int32
        L.superdc_eig_plan.argtypes = [c_void_p, ctypes.POINTER(Opts), ctypes.POINTER(c_void_p)]
        L.superdc_eig_plan.restype = c_int32
        L.superdc_eig_run.argtypes = [c_void_p, c_void_p, c_void_p]
        L.superdc_eig_run.restype = c_int32
        L.superdc_eigfact_free.argtypes = [c_void_p]
        L.superdc_eigfact_free.restype = None
        L.superdc_apply_Q.argtypes = [c_void_p, c_int32, c_int64, c_void_p, c_int64, c_void_p, c_int64, c_void_p]
        L.superdc_apply_Q.restype = c_int32
        L.superdc_apply_function.argtypes = [c_void_p, c_void_p, c_int64, c_void_p, c_int64, c_void_p, c_int64,
                                             c_void_p]
        L.superdc_apply_function.restype = c_int32
        L.superdc_eigfact_set_fmm_min_m.argtypes = [c_void_p, c_int32]
        L.superdc_eigfact_set_fmm_min_m.restype = c_int32
        L.superdc_sync_status.argtypes = [c_void_p]
        L.superdc_sync_status.restype = c_int32
        L.superdc_eigfact_stats.argtypes = [c_void_p, ctypes.POINTER(c_int64), ctypes.POINTER(c_int64),
                                            ctypes.POINTER(c_int32)]
        L.superdc_eigfact_stats.restype = c_int32
        L.superdc_eigfact_get.argtypes = [c_void_p, c_int32, c_int32, ctypes.c_char_p, c_void_p]
        L.superdc_eigfact_get.restype = c_int32
        L.superdc_eigfact_norms.argtypes = [c_void_p, ctypes.POINTER(c_double), ctypes.POINTER(c_double)]
        L.superdc_eigfact_norms.restype = c_int32
        L.superdc_eigfact_shape.argtypes = [c_void_p, ctypes.POINTER(c_int32), ctypes.POINTER(c_int32),
                                            ctypes.POINTER(c_int64)]
        L.superdc_eigfact_shape.restype = c_int32
        L.superdc_secular_batched_backward.argtypes = [c_int64, c_void_p, c_int64, c_double,
                                                       ctypes.POINTER(Rank1Out), c_void_p, c_int64, c_void_p,
                                                       c_int64, c_void_p, c_int64, c_void_p, c_void_p,
                                                       c_void_p, c_int64, c_void_p]
        L.superdc_secular_batched_backward.restype = c_int32
        L.superdc_rank1_apply.argtypes = [c_int64, c_void_p, c_int64, ctypes.POINTER(Rank1Out), c_int32, c_int64,
                                          c_void_p, c_int64, c_void_p, c_int64, ctypes.POINTER(Opts), c_void_p]
        L.superdc_rank1_apply.restype = c_int32
        L.superdc_eig_backward.argtypes = [c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_int64, c_void_p,
                                           c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int64,
                                           c_void_p]
        L.superdc_eig_backward.restype = c_int32
        L.superdc_profile_enable.argtypes = [c_int32]
        L.superdc_profile_enable.restype = c_int32
        L.superdc_profile_reset.argtypes = []
        L.superdc_profile_reset.restype = c_int32
        L.superdc_profile_read.argtypes = [ctypes.c_char_p, ctypes.POINTER(c_int64), ctypes.POINTER(c_double)]
        L.superdc_profile_read.restype = c_int32
        L.superdc_profile_counter.argtypes = [ctypes.c_char_p, ctypes.POINTER(c_int64)]
        L.superdc_profile_counter.restype = c_int32
        _lib = L
    return _lib


def check(code, where=""):
    if code != 0:
        raise SuperDCError(code, where)


def default_opts(**kw):
    o = Opts()
    check(lib().superdc_opts_default(ctypes.byref(o)), "superdc_opts_default")
    for k, v in kw.items():
        if v is not None:
            setattr(o, k, v)
    return o


def exported_symbols():
    """Names declared in include/superdc.h that the shared library must export."""
    import re
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    names = []
    for f in sorted(os.listdir(hdr)):
        if f.endswith(".h"):
            txt = open(os.path.join(hdr, f)).read()
            names += re.findall(r"^\s*(?:superdc_status|const char \*|void|superdc_\w+ \*?)\s*\*?\s*(superdc_\w+)\s*\(",
                                txt, re.M)
    return sorted(set(names))
