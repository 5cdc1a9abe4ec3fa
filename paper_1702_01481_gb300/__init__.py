"""Python binding of libblm.so, the GB300 library for one step of the blocked linear method.

Argument marshalling only: every step runs in the library's CUDA kernels.  The functions keep
the C ABI's names (include/blm.h); `Step` wraps one handle for convenience.  Arrays are torch
tensors (device or host) or anything exposing a data pointer; torch is used for memory and
streams only.  Importing this module raises if the native library has not been built: there is
no fallback.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libblm.so")

BLM_OK, BLM_ERR_ARG, BLM_ERR_STATE, BLM_ERR_NUMERIC, BLM_ERR_NOMEM, BLM_ERR_CUDA, \
    BLM_ERR_TIMEOUT, BLM_ERR_UNSUPPORTED = range(8)
BLM_PREC_F64, BLM_PREC_BF16X4, BLM_PREC_TF32X4 = 0, 1, 2
BLM_IN_F64, BLM_IN_F32 = 0, 1
STATUS_NAMES = {0: "BLM_OK", 1: "BLM_ERR_ARG", 2: "BLM_ERR_STATE", 3: "BLM_ERR_NUMERIC",
                4: "BLM_ERR_NOMEM", 5: "BLM_ERR_CUDA", 6: "BLM_ERR_TIMEOUT", 7: "BLM_ERR_UNSUPPORTED"}

if not os.path.exists(LIB_PATH):
    raise ImportError("libblm.so is not built: run `python -c 'import __graft_entry__ as g; g.build()'` "
                      "(there is no CPU fallback)")

_lib = ctypes.CDLL(LIB_PATH)


class blm_problem(ctypes.Structure):
    _fields_ = [("n_params", ctypes.c_int64),
                ("n_blocks", ctypes.c_int32),
                ("block_offsets", ctypes.POINTER(ctypes.c_int64)),
                ("n_keep", ctypes.c_int32),
                ("n_old", ctypes.c_int32),
                ("old_dirs", ctypes.c_void_p),
                ("precision", ctypes.c_int32),
                ("input_type", ctypes.c_int32),
                ("shift", ctypes.c_double),
                ("pass_samples", ctypes.c_int64)]


_H = ctypes.c_void_p
_P = ctypes.c_void_p
_sig = {
    "blm_create": (ctypes.c_int, [ctypes.POINTER(blm_problem), ctypes.c_void_p, ctypes.POINTER(_H)]),
    "blm_accumulate": (ctypes.c_int, [_H, _P, _P, _P, _P, ctypes.c_int64, ctypes.c_int64]),
    "blm_block_solve": (ctypes.c_int, [_H]),
    "blm_project": (ctypes.c_int, [_H, _P, _P, _P, _P, ctypes.c_int64, ctypes.c_int64]),
    "blm_combined_solve": (ctypes.c_int, [_H, _P, ctypes.POINTER(ctypes.c_double)]),
    "blm_get_block": (ctypes.c_int, [_H, ctypes.c_int32, _P, _P, _P, _P]),
    "blm_get_combined": (ctypes.c_int, [_H, _P, _P]),
    "blm_block_dim": (ctypes.c_int64, [_H, ctypes.c_int32]),
    "blm_combined_dim": (ctypes.c_int64, [_H]),
    "blm_reset": (ctypes.c_int, [_H]),
    "blm_destroy": (ctypes.c_int, [_H]),
    "blm_last_error": (ctypes.c_char_p, [_H]),
    "blm_set_wait_limit": (ctypes.c_int, [_H, ctypes.c_uint32]),
    "blm_set_host_cache": (ctypes.c_int, [_H, ctypes.c_size_t]),
    "blm_graph_capture": (ctypes.c_int, [_H, _P, _P, _P, _P, ctypes.c_int64, ctypes.c_int64,
                                         ctypes.c_int64, _P]),
    "blm_graph_launch": (ctypes.c_int, [_H]),
    "blm_autotune": (ctypes.c_int, [_H, _P, _P, _P, _P, ctypes.c_int64, ctypes.c_int64,
                                    ctypes.POINTER(ctypes.c_int32)]),
    "blm_set_tiles": (ctypes.c_int, [_H, ctypes.c_int32]),
    "blm_batch_create": (ctypes.c_int, [ctypes.POINTER(blm_problem), ctypes.c_int32,
                                        ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "blm_batch_capture": (ctypes.c_int, [ctypes.c_void_p, _P, _P, _P, _P, _P, _P,
                                         ctypes.c_int64, _P]),
    "blm_batch_launch": (ctypes.c_int, [ctypes.c_void_p]),
    "blm_batch_result": (ctypes.c_int, [ctypes.c_void_p, _P, _P]),
    "blm_batch_handle": (ctypes.c_void_p, [ctypes.c_void_p, ctypes.c_int32]),
    "blm_batch_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "blm_batch_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "blm_graph_result": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_double)]),
    "blm_memory_estimate": (ctypes.c_size_t, [ctypes.POINTER(blm_problem)]),
    "blm_lm_matrix_bytes": (ctypes.c_double, [ctypes.c_int64]),
    "blm_matrix_bytes_dominant": (ctypes.c_double, [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32]),
    "blm_profile": (ctypes.c_int, [_H, ctypes.c_int]),
    "blm_profile_read": (ctypes.c_int, [_H, ctypes.c_int, _P, _P]),
    "blm_profile_class_name": (ctypes.c_char_p, [ctypes.c_int]),
    "blm_noalloc_max_dim": (ctypes.c_int32, []),
    "blm_block_solve_noalloc": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_int32, _P, _P,
                                               ctypes.c_void_p]),
}
BLM_PROF_CLASSES = 14
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_sig)


class BLMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


def _ptr(x):
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    if hasattr(x, "ctypes"):
        return ctypes.c_void_p(x.ctypes.data)
    return ctypes.c_void_p(int(x))


def make_problem(n_params, block_offsets, n_keep, n_old=0, old_dirs=None,
                 precision=BLM_PREC_F64, input_type=BLM_IN_F64, shift=0.0, pass_samples=0):
    offs = (ctypes.c_int64 * len(block_offsets))(*[int(o) for o in block_offsets])
    p = blm_problem(int(n_params), len(block_offsets) - 1, offs, int(n_keep), int(n_old),
                    _ptr(old_dirs), int(precision), int(input_type), float(shift),
                    int(pass_samples))
    p._keep = (offs, old_dirs)          # keep the arrays alive with the struct
    return p


# ----- the C ABI under its own names ---------------------------------------------------------
def blm_create(problem, stream=0):
    h = _H()
    st = _lib.blm_create(ctypes.byref(problem), ctypes.c_void_p(int(stream)), ctypes.byref(h))
    if st != BLM_OK:
        raise BLMError(st, "blm_create failed")
    return h


def _check(h, st, what):
    if st != BLM_OK:
        raise BLMError(st, "%s: %s" % (what, _lib.blm_last_error(h).decode()))


def blm_accumulate(h, O, dEL, EL, w, n_samples, ld):
    _check(h, _lib.blm_accumulate(h, _ptr(O), _ptr(dEL), _ptr(EL), _ptr(w), int(n_samples), int(ld)),
           "blm_accumulate")


def blm_block_solve(h):
    _check(h, _lib.blm_block_solve(h), "blm_block_solve")


def blm_project(h, O, dEL, EL, w, n_samples, ld):
    _check(h, _lib.blm_project(h, _ptr(O), _ptr(dEL), _ptr(EL), _ptr(w), int(n_samples), int(ld)),
           "blm_project")


def blm_combined_solve(h, dmu):
    e = ctypes.c_double()
    _check(h, _lib.blm_combined_solve(h, _ptr(dmu), ctypes.byref(e)), "blm_combined_solve")
    return e.value


def blm_get_block(h, b, S=None, H=None, lam=None, B=None):
    _check(h, _lib.blm_get_block(h, int(b), _ptr(S), _ptr(H), _ptr(lam), _ptr(B)), "blm_get_block")


def blm_get_combined(h, S=None, H=None):
    _check(h, _lib.blm_get_combined(h, _ptr(S), _ptr(H)), "blm_get_combined")


def blm_block_dim(h, b):
    return int(_lib.blm_block_dim(h, int(b)))


def blm_combined_dim(h):
    return int(_lib.blm_combined_dim(h))


def blm_reset(h):
    _check(h, _lib.blm_reset(h), "blm_reset")


def blm_destroy(h):
    _lib.blm_destroy(h)


def blm_last_error(h):
    return _lib.blm_last_error(h).decode()


def blm_set_host_cache(h, nbytes):
    _check(h, _lib.blm_set_host_cache(h, int(nbytes)), "blm_set_host_cache")


BLM_WAIT_LIMIT_DEFAULT = 1 << 24


def blm_set_wait_limit(h, polls):
    _check(h, _lib.blm_set_wait_limit(h, int(polls)), "blm_set_wait_limit")


def blm_graph_capture(h, O, dEL, EL, w, n_samples, chunk, ld, dmu):
    _check(h, _lib.blm_graph_capture(h, _ptr(O), _ptr(dEL), _ptr(EL), _ptr(w), int(n_samples),
                                     int(chunk), int(ld), _ptr(dmu)), "blm_graph_capture")


def blm_autotune(h, O, dEL, EL, w, n_samples, ld):
    """Chooses the tile layout and work-unit length for the handle; returns the choice index."""
    c = ctypes.c_int32()
    _check(h, _lib.blm_autotune(h, _ptr(O), _ptr(dEL), _ptr(EL), _ptr(w), int(n_samples), int(ld),
                                ctypes.byref(c)), "blm_autotune")
    return c.value


def blm_set_tiles(h, choice):
    _check(h, _lib.blm_set_tiles(h, int(choice)), "blm_set_tiles")


def blm_graph_launch(h):
    _check(h, _lib.blm_graph_launch(h), "blm_graph_launch")


def blm_graph_result(h):
    e = ctypes.c_double()
    _check(h, _lib.blm_graph_result(h, ctypes.byref(e)), "blm_graph_result")
    return e.value


def _bcheck(b, st, what):
    if st != BLM_OK:
        raise BLMError(st, "%s: %s" % (what, _lib.blm_batch_last_error(b).decode()))


def blm_batch_create(problems, stream=0):
    arr = (blm_problem * len(problems))(*problems)
    b = ctypes.c_void_p()
    st = _lib.blm_batch_create(arr, len(problems), ctypes.c_void_p(int(stream)), ctypes.byref(b))
    if st != BLM_OK:
        raise BLMError(st, "blm_batch_create failed")
    return b


def _ptr_array(xs):
    return (ctypes.c_void_p * len(xs))(*[None if x is None else _ptr(x).value for x in xs])


def blm_batch_capture(b, O, dEL, EL, w, n_samples, ld, chunk, dmu):
    """Lists of per-problem device arrays (w may be None or a list with None entries)."""
    k = len(O)
    ns = (ctypes.c_int64 * k)(*[int(x) for x in n_samples])
    lds = (ctypes.c_int64 * k)(*[int(x) for x in ld])
    wp = None if w is None else _ptr_array(w)
    _bcheck(b, _lib.blm_batch_capture(b, _ptr_array(O), _ptr_array(dEL), _ptr_array(EL), wp, ns,
                                      lds, int(chunk), _ptr_array(dmu)), "blm_batch_capture")


def blm_batch_launch(b):
    _bcheck(b, _lib.blm_batch_launch(b), "blm_batch_launch")


def blm_batch_result(b, count):
    """(predicted energies, statuses) of the last launch; raises on the first failure."""
    import numpy as np
    e = np.empty(count)
    st = np.empty(count, dtype=np.int32)
    r = _lib.blm_batch_result(b, _ptr(e), _ptr(st))
    return e, st, r


def blm_batch_handle(b, i):
    return _H(_lib.blm_batch_handle(b, int(i)))


def blm_batch_destroy(b):
    _lib.blm_batch_destroy(b)


def blm_memory_estimate(problem):
    return int(_lib.blm_memory_estimate(ctypes.byref(problem)))


def blm_lm_matrix_bytes(n_params):
    return float(_lib.blm_lm_matrix_bytes(int(n_params)))


def blm_matrix_bytes_dominant(n_params, n_blocks, n_old):
    return float(_lib.blm_matrix_bytes_dominant(int(n_params), int(n_blocks), int(n_old)))


def blm_profile(h, enable):
    _check(h, _lib.blm_profile(h, int(enable)), "blm_profile")


def blm_profile_read(h):
    """{class name: (milliseconds, launches)} since the last blm_profile(h, 1)."""
    ms = (ctypes.c_double * BLM_PROF_CLASSES)()
    n = (ctypes.c_int64 * BLM_PROF_CLASSES)()
    _check(h, _lib.blm_profile_read(h, BLM_PROF_CLASSES, ms, n), "blm_profile_read")
    return {_lib.blm_profile_class_name(i).decode(): (ms[i], n[i]) for i in range(BLM_PROF_CLASSES)}


def blm_noalloc_max_dim():
    return int(_lib.blm_noalloc_max_dim())


def blm_block_solve_noalloc(S, H, dim, n_keep, lam, B, stream=0):
    """One block problem through the allocation-free entry point (device arrays)."""
    st = _lib.blm_block_solve_noalloc(_ptr(S), _ptr(H), int(dim), int(n_keep), _ptr(lam), _ptr(B),
                                      ctypes.c_void_p(int(stream)))
    if st != BLM_OK:
        raise BLMError(st, "blm_block_solve_noalloc")


# ----- convenience wrapper ---------------------------------------------------------------------
class Step:
    """One BLM step on one handle.  Sample tensors: O, dEL (ns x ld), EL, w (ns), all of the
    problem's input dtype, on the device or on the host."""

    def __init__(self, n_params, block_offsets, n_keep, n_old=0, old_dirs=None,
                 precision=BLM_PREC_F64, input_type=BLM_IN_F64, shift=0.0, stream=0,
                 pass_samples=0):
        self.problem = make_problem(n_params, block_offsets, n_keep, n_old, old_dirs, precision,
                                    input_type, shift, pass_samples)
        self.n = int(n_params)
        self.offsets = [int(o) for o in block_offsets]
        self.n_keep = int(n_keep)
        self.h = blm_create(self.problem, stream)

    def accumulate(self, O, dEL, EL, w=None):
        blm_accumulate(self.h, O, dEL, EL, w, O.shape[0], O.stride(0) if hasattr(O, "stride") else O.shape[1])

    def block_solve(self):
        blm_block_solve(self.h)

    def project(self, O, dEL, EL, w=None):
        blm_project(self.h, O, dEL, EL, w, O.shape[0], O.stride(0) if hasattr(O, "stride") else O.shape[1])

    def combined_solve(self, dmu):
        return blm_combined_solve(self.h, dmu)

    def block(self, b):
        """(S, H, lambda, B) of block b as numpy arrays."""
        import numpy as np
        d = blm_block_dim(self.h, b)
        m = self.offsets[b + 1] - self.offsets[b]
        k = min(self.n_keep, m)
        S = np.empty((d + 1, d + 1))
        H = np.empty((d + 1, d + 1))
        lam = np.empty(k)
        B = np.empty((k, m))
        blm_get_block(self.h, b, S, H, lam, B)
        return S, H, lam, B

    def combined(self):
        import numpy as np
        d = blm_combined_dim(self.h)
        S = np.empty((d + 1, d + 1))
        H = np.empty((d + 1, d + 1))
        blm_get_combined(self.h, S, H)
        return S, H

    def reset(self):
        blm_reset(self.h)

    def close(self):
        if self.h:
            blm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
