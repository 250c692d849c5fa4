"""ctypes loader for librsk.so and its C signatures (argument marshalling only).

The library is built in-tree by ``paper_2508_21189_gb300.build`` (``__graft_entry__.build()``).
If it is missing this module raises: there is no fallback implementation.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librsk.so")

STATUS = {0: "RSK_OK", 1: "RSK_ERR_INVALID_ARG", 2: "RSK_ERR_NOMEM", 3: "RSK_ERR_CUDA",
          4: "RSK_ERR_NOT_CONVERGED", 5: "RSK_ERR_TIMEOUT", 6: "RSK_ERR_UNSUPPORTED",
          7: "RSK_ERR_INTERNAL"}

c_i32, c_i64, c_u64, c_p, c_f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_double

# name -> argument types (all functions return rsk_status as int32 unless listed in _RESTYPE)
SIGNATURES = {
    "rsk_create": [c_p],
    "rsk_destroy": [c_p],
    "rsk_last_error": [c_p],
    "rsk_sync_status": [c_p, c_p],
    "rsk_version": [],
    "rsk_set_wait_limit": [c_p, ctypes.c_uint32],
    "rsk_profile_enable": [c_p, c_i32],
    "rsk_profile_read": [c_p, c_i32, c_p, c_p],
    "rsk_sparse_sign_generate": [c_p, c_i64, c_i64, c_i32, c_u64, c_p, c_p, c_p],
    "rsk_sparse_sign_index_dims": [c_i64, c_i64, c_i32, c_p, c_p, c_p],
    "rsk_sparse_sign_index": [c_p, c_i64, c_i64, c_i32, c_u64, c_p, c_p, c_p],
    "rsk_sparse_sign_apply": [c_p, c_p, c_i32, c_i64, c_i64, c_i64, c_i64, c_i32, c_u64, c_p, c_i32, c_i64, c_p],
    "rsk_sparse_sign_apply_rows": [c_p, c_p, c_i32, c_i64, c_i64, c_i64, c_i64, c_i64, c_i32, c_u64, c_p, c_i32, c_i64,
                                   c_p],
    "rsk_sketch_sum_partials": [c_p, c_p, c_i32, c_i32, c_i64, c_i64, c_i64, c_p, c_i64, c_p],
    "rsk_srtt_apply_rows": [c_p, c_p, c_i32, c_i64, c_i64, c_i64, c_i64, c_i64, c_i64, c_u64, c_p, c_i32, c_i64, c_p],
    "rsk_sparse_sign_apply_noalloc": [c_p, c_i32, c_i64, c_i64, c_i64, c_i64, c_i32, c_u64, c_p, c_i32, c_i64, c_p],
    "rsk_sparse_sign_apply_host": [c_p, c_p, c_i32, c_i64, c_i64, c_i64, c_i64, c_i32, c_u64, c_p, c_i32, c_i64, c_p],
    "rsk_sparse_stack_generate": [c_p, c_i64, c_i64, c_i32, c_u64, c_p, c_p, c_p],
    "rsk_sparse_stack_apply": [c_p, c_p, c_i32, c_i64, c_i64, c_i64, c_i64, c_i32, c_u64, c_p, c_i32, c_i64, c_p],
    "rsk_sparse_sign_apply_right": [c_p, c_i32, c_p, c_i64, c_i64, c_i64, c_i64, c_i32, c_u64, c_i32, c_p, c_i64,
                                    c_p],
    "rsk_sparse_sign_plan_create": [c_p, c_i64, c_i64, c_i32, c_u64, c_p, c_p],
    "rsk_sparse_sign_plan_apply": [c_p, c_p, c_p, c_i32, c_i64, c_i64, c_p, c_i32, c_i64, c_p],
    "rsk_sparse_sign_plan_destroy": [c_p, c_p, c_p],
    "rsk_srtt_draw": [c_p, c_i64, c_i64, c_u64, c_p, c_p, c_p],
    "rsk_srtt_apply": [c_p, c_p, c_i32, c_i64, c_i64, c_i64, c_i64, c_u64, c_p, c_i32, c_i64, c_p],
    "rsk_sparse_rtt_default_xi": [c_i64],
    "rsk_sparse_rtt_draw": [c_p, c_i64, c_i64, c_i32, c_u64, c_p, c_p, c_p],
    "rsk_sparse_rtt_apply": [c_p, c_p, c_i32, c_i64, c_i64, c_i64, c_i64, c_i32, c_u64, c_p, c_i32, c_i64, c_p],
    "rsk_split_pairs": [c_p, c_p, c_i64, c_i64, c_i64, c_p, c_p],
    "rsk_lstsq_sketch_precond": [c_p, c_p, c_i32, c_i64, c_i64, c_i64, c_p, c_p, c_p, c_p, c_p],
    "rsk_lstsq_sketch_precond_batched": [c_p, c_i32, c_p, c_p, c_p, c_p],
    "rsk_svd_econ": [c_p, c_p, c_i64, c_i64, c_i64, c_p, c_i64, c_p, c_p, c_i64, c_p],
    "rsk_qr_econ": [c_p, c_p, c_i64, c_i64, c_i64, c_p, c_i64, c_p, c_p],
    "rsk_cholesky": [c_p, c_p, c_i64, c_i64, ctypes.c_float, c_p, c_i64, c_p],
    "rsk_trinv": [c_p, c_p, c_i64, c_i64, c_p, c_p],
    "rsk_nystrom_psd": [c_p, c_p, c_i64, c_i64, c_i32, c_i32, c_i32, c_u64, c_i32, c_p, c_i64, c_p, c_p],
    "rsk_gen_nystrom": [c_p, c_p, c_i64, c_i64, c_i64, c_i32, c_i32, c_i32, c_u64, c_i32, c_i32, c_p, c_i64, c_p, c_p,
                        c_i64, c_p, c_p],
    "rsk_osi_estimate": [c_p, c_i64, c_i64, c_i32, c_u64, c_i32, c_i32, c_p, c_p, c_p],
    "rsk_tune_cache_load": [ctypes.c_char_p],
    "rsk_tune_cache_save": [ctypes.c_char_p],
    "rsk_tune_cache_clear": [],
    "rsk_tune_cache_set": [c_i32, c_i32, c_i64, c_i64, c_i64, c_i32, c_i32],
    "rsk_tune_cache_get": [c_i32, c_i32, c_i64, c_i64, c_i64, c_i32, c_p],
    "rsk_autotune_sketch": [c_p, c_i32, c_i32, c_i64, c_i64, c_i64, c_i32, c_p, c_p, c_p],
    "rsk_autotune_batched": [c_p, c_i32, c_p, c_p, c_p, c_p, c_p],
    "rsk_gemm_bf16": [c_p, c_p, c_i64, c_i64, c_i64, c_p, c_i64, c_i64, c_p, c_i64, c_i32, c_p],
    "rsk_gemm_bf16_ex": [c_p, c_i32, c_p, c_i64, c_i64, c_i64, c_p, c_i64, c_i64, c_p, c_i64, c_i32, c_i32, c_i32,
                         c_p],
    "rsk_gemm_f32": [c_p, c_i32, c_p, c_i64, c_i64, c_i64, c_p, c_i64, c_i64, c_p, c_i64, c_i32, c_i32, c_p],
    "rsk_rsvd": [c_p, c_p, c_i64, c_i64, c_i64, c_i32, c_i32, c_i32, c_u64, c_p, c_p, c_p, c_p],
}


class LsqProblem(ctypes.Structure):
    """rsk_lsq_problem (rsk.h)."""
    _fields_ = [("A", ctypes.c_void_p), ("a_dtype", ctypes.c_int32), ("n", ctypes.c_int64), ("k", ctypes.c_int64),
                ("lda", ctypes.c_int64), ("d", ctypes.c_int64), ("b", ctypes.c_void_p), ("x", ctypes.c_void_p)]


class LsqOpts(ctypes.Structure):
    """rsk_lsq_opts (rsk.h)."""
    _fields_ = [("d", ctypes.c_int64), ("zeta", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("sketch_dtype", ctypes.c_int32), ("inner_dtype", ctypes.c_int32),
                ("tol_backward", ctypes.c_double), ("max_refine", ctypes.c_int32),
                ("max_inner_iters", ctypes.c_int32), ("inner_tol", ctypes.c_double),
                ("qr_dtype", ctypes.c_int32)]


class LsqInfo(ctypes.Structure):
    """rsk_lsq_info (rsk.h)."""
    _fields_ = [("backward_err", ctypes.c_double), ("residual_norm", ctypes.c_double),
                ("frobenius_norm", ctypes.c_double), ("refine_steps", ctypes.c_int32),
                ("inner_iters", ctypes.c_int32), ("status", ctypes.c_int32)]
_RESTYPE = {"rsk_last_error": ctypes.c_char_p}

_lib = None


def load():
    """Load librsk.so (once) and attach the C signatures.  Raises if it was not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"librsk.so not found at {LIB_PATH}; run __graft_entry__.build() "
                          "(there is no fallback implementation)")
    lib = ctypes.CDLL(LIB_PATH)
    for name, args in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = _RESTYPE.get(name, ctypes.c_int32)
    _lib = lib
    return lib


class RskError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status
