"""ctypes binding of libsfft.so (include/sfft.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts torch tensors to device
pointers, fills the C structs and raises SfftError on a non-zero status.  Importing it
raises ImportError when libsfft.so has not been built (no fallback exists).
"""
from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsfft.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first "
                      "(python -c 'import __graft_entry__ as g; g.build()')")

lib = C.CDLL(LIB_PATH)

# status codes / enums (include/sfft.h)
OK, EINVAL, ENOTPRIME, EALIAS, EOVERFLOW, ENOMEM, ECUDA, ETIMEOUT, ECAPACITY, ESTATE = range(10)
FP64, FP32 = 0, 1
L_COR26, L_EQ42, L_FALLBACK = 0, 1, 2
COMBINE_MEDIAN, COMBINE_HYBRID, COMBINE_LSQ = 0, 1, 2

_NAMES = {0: "SFFT_OK", 1: "SFFT_EINVAL", 2: "SFFT_ENOTPRIME", 3: "SFFT_EALIAS", 4: "SFFT_EOVERFLOW",
          5: "SFFT_ENOMEM", 6: "SFFT_ECUDA", 7: "SFFT_ETIMEOUT", 8: "SFFT_ECAPACITY", 9: "SFFT_ESTATE"}


class SfftError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


CAND_I32, CAND_I8 = 0, 1
DFT_DF64, DFT_FP32 = 0, 1


class Params(C.Structure):
    _fields_ = [("c", C.c_double), ("delta", C.c_double), ("nu", C.c_double), ("tau_abs", C.c_double),
                ("tau_rel", C.c_double), ("theta_abs", C.c_double), ("theta_rel", C.c_double),
                ("s_tilde", C.c_int64), ("precision", C.c_int), ("refine", C.c_int), ("L_rule", C.c_int),
                ("combine", C.c_int), ("seed", C.c_uint64), ("detect_cap", C.c_int64), ("cand_type", C.c_int),
                ("cand_ld", C.c_int), ("dft", C.c_int), ("rank_bits", C.c_int)]


class Diag(C.Structure):
    _fields_ = [("counts", C.c_void_p), ("hashes", C.c_void_p), ("collisions", C.c_void_p),
                ("detected", C.c_void_p), ("pcheck", C.c_void_p), ("ghat", C.c_void_p), ("tau", C.c_void_p),
                ("n_detected", C.c_int64), ("n_guard", C.c_int64), ("lsq_iters", C.c_int64)]


class DimIncrParams(C.Structure):
    _fields_ = [("s", C.c_int64), ("s_local", C.c_int64), ("r", C.c_int), ("theta_abs", C.c_double),
                ("theta_rel", C.c_double), ("delta", C.c_double), ("c", C.c_double), ("tau_abs", C.c_double),
                ("tau_rel", C.c_double), ("precision", C.c_int), ("refine", C.c_int), ("seed", C.c_uint64),
                ("max_samples", C.c_int64), ("rank_bits", C.c_int), ("L_rule", C.c_int)]


class SparsePolyCtx(C.Structure):
    _fields_ = [("kvec", C.c_void_p), ("coef", C.c_void_p), ("n_terms", C.c_int64), ("d", C.c_int)]


class BsplineCtx(C.Structure):
    _fields_ = [("dims", C.c_void_p), ("orders", C.c_void_p), ("n_terms", C.c_int), ("d", C.c_int)]


class SopCtx(C.Structure):
    _fields_ = [("triples", C.c_void_p), ("theta", C.c_void_p), ("n_terms", C.c_int), ("K", C.c_int),
                ("width", C.c_double), ("d", C.c_int), ("work", C.c_void_p)]


SAMPLE_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p)

_vp, _i64, _i32, _dbl = C.c_void_p, C.c_int64, C.c_int, C.c_double
_P = C.POINTER


def _sig(name, res, args):
    f = getattr(lib, name)
    f.restype = res
    f.argtypes = args
    return f


sfft_params_default = _sig("sfft_params_default", None, [_P(Params)])
sfft_plan_create = _sig("sfft_plan_create", _i32, [_P(_vp), _i32, _vp, _i64, _i64, _i32, _vp, _vp, _P(Params), _vp])
sfft_plan_set_candidates = _sig("sfft_plan_set_candidates", _i32, [_vp, _vp, _i64])
sfft_plan_set_generators = _sig("sfft_plan_set_generators", _i32, [_vp, _vp])
sfft_plan_info = _sig("sfft_plan_info", _i32, [_vp, _P(_i32), _vp, _vp, _P(_i64)])
sfft_plan_destroy = _sig("sfft_plan_destroy", None, [_vp])
sfft_sample_points = _sig("sfft_sample_points", _i32, [_vp, _vp, _vp, _vp])
sfft_reconstruct = _sig("sfft_reconstruct", _i32, [_vp, _vp, _vp, _vp, _i64, _P(_i64), _P(Diag)])
sfft_reconstruct_shard_begin = _sig("sfft_reconstruct_shard_begin", _i32, [_vp, _vp, _vp, _P(_i64)])
sfft_reconstruct_shard_end = _sig("sfft_reconstruct_shard_end", _i32, [_vp, _vp, _vp, _vp, _vp, _i64, _P(_i64)])
sfft_reconstruct_backward = _sig("sfft_reconstruct_backward", _i32, [_vp, _vp, _vp])
sfft_sample_sparse_poly = _sig("sfft_sample_sparse_poly", _i32, [_vp, _vp, _vp, _i64, _vp, _vp])
sfft_sample_sop = _sig("sfft_sample_sop", _i32, [_vp, _vp, _vp, _i32, _i32, _dbl, _vp])
sfft_sample_bspline = _sig("sfft_sample_bspline", _i32, [_vp, _vp, _vp, _i32, _vp])
sfft_sample_sop_backward = _sig("sfft_sample_sop_backward", _i32, [_vp, _vp, _vp, _i32, _i32, _dbl, _vp, _vp])
sfft_batch_create = _sig("sfft_batch_create", _i32, [_P(_vp), _vp, _i32, _i32, _vp])
sfft_batch_destroy = _sig("sfft_batch_destroy", None, [_vp])
sfft_batch_reconstruct = _sig("sfft_batch_reconstruct", _i32, [_vp, _vp, _vp, _vp, _vp, _vp])
sfft_batch_sample_sparse_poly = _sig("sfft_batch_sample_sparse_poly", _i32, [_vp, _vp, _vp, _vp, _vp, _vp])
sfft_batch_autotune = _sig("sfft_batch_autotune", _i32, [_vp, _vp, _vp, _vp, _vp, _i32, _P(_dbl), _P(_i32)])
sfft_batch_select_hash = _sig("sfft_batch_select_hash", _i32, [_vp, _i32])
sfft_batch_set_shapes = _sig("sfft_batch_set_shapes", _i32, [_vp, _dbl, _i32])
sfft_batch_launch_count = _sig("sfft_batch_launch_count", _i32, [_vp, _P(_i32), _P(_i32)])
sfft_batch_flags = _sig("sfft_batch_flags", _i32, [_vp, _vp])
sfft_batch_timing = _sig("sfft_batch_timing", _i32, [_vp, _i32, _vp, _vp])
STAGES = ["clear", "fft_fwd", "zero_test", "hash_count", "compact", "det_hashes", "combine", "lsq", "refine_scatter",
          "refine_update", "select"]
sfft_dimincr_params_default = _sig("sfft_dimincr_params_default", None, [_P(DimIncrParams)])
sfft_dim_incremental = _sig("sfft_dim_incremental", _i32,
                            [_i32, _vp, _vp, _P(DimIncrParams), _vp, _vp, _vp, _vp, _i64, _P(_i64), _P(_i64), _vp])
sfft_fn_sparse_poly = _sig("sfft_fn_sparse_poly", _i32, [_vp, _vp, _i64, _vp, _vp])
sfft_fn_sop = _sig("sfft_fn_sop", _i32, [_vp, _vp, _i64, _vp, _vp])
sfft_fn_bspline = _sig("sfft_fn_bspline", _i32, [_vp, _vp, _i64, _vp, _vp])
sfft_detect_noalloc = _sig("sfft_detect_noalloc", _i32, [_i32, _vp, _i64, _i32, _vp, _vp, _vp, _vp, _dbl, _vp, _i64,
                                                        _P(_i64), _vp])
sfft_philox4x64_word0 = _sig("sfft_philox4x64_word0", C.c_uint64, [C.c_uint64] * 5)
sfft_next_prime_above = _sig("sfft_next_prime_above", _i64, [_dbl])
sfft_L_rule = _sig("sfft_L_rule", _i32, [_i32, _i64, _dbl, _dbl])
sfft_last_error = _sig("sfft_last_error", C.c_char_p, [])


def check(rc):
    if rc != OK:
        raise SfftError(rc, sfft_last_error().decode())
    return rc


def default_params(**kw) -> Params:
    p = Params()
    sfft_params_default(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def default_dimincr_params(**kw) -> DimIncrParams:
    p = DimIncrParams()
    sfft_dimincr_params_default(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def fn_address(name: str) -> int:
    """Address of a built-in black-box sample function (sfft_fn_sparse_poly / sfft_fn_sop)."""
    return C.cast(getattr(lib, name), C.c_void_p).value
