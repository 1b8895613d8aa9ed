"""Python binding of libkpp (include/kpp.h): argument marshalling through ctypes, nothing else.

Every step of the solver runs in the CUDA library.  There is no CPU fallback: if ``libkpp.so`` is
missing or cannot be loaded, every call raises ``RuntimeError``.  PyTorch tensors provide device
memory and streams; their data pointers are passed straight through the C ABI.

Paper: Derezinski, Needell, Rebrova, Yang, "Randomized Kaczmarz Methods with Beyond-Krylov
Convergence" (arXiv 2501.11673).  ``kpp_solve`` is Kaczmarz++ (Alg. 1 / Alg. 5 with exact memoised
projections); ``cdpp_solve`` is CD++ (Eq. 5.1, Alg. 3); ``kpp_factor_blocks`` memoises the block
factors (Sec. 4, Sec. 5.2).
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libkpp.so")

KPP_F64, KPP_F32, KPP_BF16 = 0, 1, 2
STATUS = {0: "KPP_OK", 1: "KPP_ERR_ARG", 2: "KPP_ERR_CUDA", 3: "KPP_ERR_OOM", 4: "KPP_ERR_NOT_SPD",
          5: "KPP_ERR_NUMERIC", 6: "KPP_ERR_NO_CONVERGENCE", 7: "KPP_ERR_TIMEOUT", 8: "KPP_ERR_BUDGET",
          9: "KPP_ERR_UNSUPPORTED"}
OK, ERR_ARG, ERR_CUDA, ERR_OOM, ERR_NOT_SPD, ERR_NUMERIC, ERR_NO_CONVERGENCE, ERR_TIMEOUT, ERR_BUDGET, \
    ERR_UNSUPPORTED = range(10)

# Every symbol include/kpp.h declares (checked by the CPU test suite against the built library).
EXPORTS = ["kpp_params_default", "kpp_status_string", "kpp_last_error", "kpp_partition", "kpp_partition_destroy",
           "kpp_partition_blocks", "kpp_factor_blocks", "kpp_factors_destroy", "kpp_factors_bad_block", "kpp_factors_fp64_blocks", "kpp_factors_stage_ms", "kpp_factors_get_memo",
           "kpp_factors_get_block", "kpp_solve", "cdpp_solve", "kpp_solve_host", "kpp_rel_residual",
           "kpp_solve_batched", "kpp_sample_blocks", "cdpp_solve_noalloc", "kpp_set_kernel_variant", "kpp_set_wait_test", "kpp_block_gram", "kpp_server_create", "kpp_server_add_matrix",
           "kpp_server_submit", "kpp_server_poll", "kpp_server_wait_all", "kpp_server_stats", "kpp_server_reset_stats", "kpp_server_destroy",
           "cdpp_solve_batched", "kpp_plan_create", "kpp_plan_launch", "kpp_plan_report", "kpp_plan_info",
           "kpp_plan_destroy", "kpp_tune_cache_size", "kpp_tune_cache_clear", "kpp_tune_cache_save",
           "kpp_tune_cache_load", "kpp_launch_count", "kpp_device_alloc_count", "kpp_device_cache_bytes", "kpp_device_cache_trim", "kpp_build_info", "kpp_rht_forward", "kpp_rht_inverse",
           "kpp_memo_sequence", "kpp_state_create", "kpp_state_destroy", "kpp_state_step",
           "kpp_state_bytes", "kpp_state_save", "kpp_state_load", "kpp_solve_resume", "cdpp_solve_resume", "kpp_cg", "kpp_gmres", "kpp_tune_block_size", "kpp_solve_memo", "kpp_factor_lsqr", "kpp_proj_lsqr", "kpp_solve_lsqr"]
GRID_TUNE = -1  # Params.grid: let the launch autotuner choose the CTAs per system


class KppError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Matrix(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("dtype", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("rows", ctypes.c_int64), ("cols", ctypes.c_int64), ("ld", ctypes.c_int64)]


class Params(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("tol", ctypes.c_double), ("max_iters", ctypes.c_int64),
                ("seed", ctypes.c_uint64), ("sys_id", ctypes.c_uint32), ("adaptive_rho", ctypes.c_int32),
                ("rho0", ctypes.c_double), ("eta", ctypes.c_double), ("grid", ctypes.c_int32),
                ("refine", ctypes.c_int32), ("max_outer", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("inner_tol", ctypes.c_double), ("reserved1", ctypes.c_int64 * 4)]


class ServingStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("failed", ctypes.c_int64), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double), ("solves_per_s", ctypes.c_double),
                ("span_s", ctypes.c_double), ("peak_bytes", ctypes.c_size_t), ("budget_bytes", ctypes.c_size_t),
                ("loop_launches", ctypes.c_int64), ("loop_slots", ctypes.c_int64), ("reserved", ctypes.c_int64 * 2)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class Report(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64), ("outer", ctypes.c_int64), ("rel_res_true", ctypes.c_double),
                ("rel_res_est", ctypes.c_double), ("rho_final", ctypes.c_double), ("status", ctypes.c_int32),
                ("bad_block", ctypes.c_int32), ("device_ms", ctypes.c_double), ("kernel_ms", ctypes.c_double),
                ("launches", ctypes.c_int64), ("reserved", ctypes.c_int64 * 2)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


_lib = None
_lock = threading.Lock()


def load(path: str | None = None):
    """Load libkpp.so (built by ``paper_2501_11673_gb300.build``).  Raises if it is absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libkpp.so not found at {p}: build it with paper_2501_11673_gb300.build.build()")
        lib = ctypes.CDLL(p)
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        lib.kpp_params_default.restype = Params
        lib.kpp_status_string.argtypes = [ctypes.c_int]
        lib.kpp_status_string.restype = ctypes.c_char_p
        lib.kpp_last_error.restype = ctypes.c_char_p
        lib.kpp_build_info.restype = ctypes.c_char_p
        lib.kpp_partition.argtypes = [i64, i32, ctypes.POINTER(vp)]
        lib.kpp_partition_destroy.argtypes = [vp]
        lib.kpp_partition_blocks.argtypes = [vp]
        lib.kpp_partition_blocks.restype = i64
        lib.kpp_factor_blocks.argtypes = [ctypes.POINTER(Matrix), vp, dbl, i32, ctypes.POINTER(vp), vp]
        lib.kpp_factors_destroy.argtypes = [vp]
        lib.kpp_factors_bad_block.argtypes = [vp]
        lib.kpp_factors_bad_block.restype = i64
        lib.kpp_factors_fp64_blocks.argtypes = [vp]
        lib.kpp_factors_fp64_blocks.restype = i64
        lib.kpp_factors_stage_ms.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
        lib.kpp_factors_stage_ms.restype = ctypes.c_int
        lib.kpp_factors_get_memo.argtypes = [vp, i64, i64, ctypes.POINTER(ctypes.c_float)]
        lib.kpp_factors_get_memo.restype = ctypes.c_int
        lib.kpp_factors_get_block.argtypes = [vp, i64, ctypes.POINTER(ctypes.c_double)]
        for name in ("kpp_solve", "cdpp_solve", "cdpp_solve_noalloc"):
            f = getattr(lib, name)
            f.argtypes = [ctypes.POINTER(Matrix), vp, vp, vp, vp, ctypes.POINTER(Params), ctypes.POINTER(Report), vp]
        lib.kpp_solve_host.argtypes = [ctypes.POINTER(Matrix), vp, vp, i32, i32, ctypes.POINTER(Params),
                                       ctypes.POINTER(Report), vp]
        lib.kpp_rel_residual.argtypes = [ctypes.POINTER(Matrix), vp, vp, ctypes.POINTER(ctypes.c_double), vp]
        lib.kpp_solve_batched.argtypes = [i32, ctypes.POINTER(Matrix), ctypes.POINTER(vp), ctypes.POINTER(vp), i32,
                                          vp, ctypes.POINTER(vp), ctypes.POINTER(Params), ctypes.POINTER(Report), vp]
        lib.kpp_sample_blocks.argtypes = [ctypes.c_uint64, ctypes.c_uint32, i64, i64, i32, vp, vp]
        lib.cdpp_solve_batched.argtypes = lib.kpp_solve_batched.argtypes
        lib.cdpp_solve_batched.restype = ctypes.c_int
        lib.kpp_set_kernel_variant.argtypes = [i32]
        lib.kpp_set_wait_test.argtypes = [ctypes.c_uint64, i32]
        lib.kpp_server_create.argtypes = [ctypes.c_size_t, i32, i32, ctypes.POINTER(vp)]
        lib.kpp_server_add_matrix.argtypes = [vp, ctypes.POINTER(Matrix), i32, dbl, i32, ctypes.POINTER(i32)]
        lib.kpp_server_submit.argtypes = [vp, i32, vp, i32, ctypes.POINTER(Params), ctypes.POINTER(i64)]
        lib.kpp_server_poll.argtypes = [vp, i64, vp, ctypes.POINTER(Report), ctypes.POINTER(i32)]
        lib.kpp_server_wait_all.argtypes = [vp, dbl]
        lib.kpp_server_stats.argtypes = [vp, ctypes.POINTER(ServingStats)]
        lib.kpp_server_destroy.argtypes = [vp]
        lib.kpp_server_reset_stats.argtypes = [vp]
        lib.kpp_server_reset_stats.restype = ctypes.c_int
        for name in ("kpp_server_create", "kpp_server_add_matrix", "kpp_server_submit", "kpp_server_poll",
                     "kpp_server_wait_all", "kpp_server_stats"):
            getattr(lib, name).restype = ctypes.c_int
        lib.kpp_block_gram.argtypes = [ctypes.POINTER(Matrix), i32, dbl, i32, vp, ctypes.POINTER(i32), vp]
        lib.kpp_block_gram.restype = ctypes.c_int
        lib.kpp_rht_forward.argtypes = [i64, vp, ctypes.POINTER(Matrix), vp, vp, vp, i32, vp]
        lib.kpp_rht_forward.restype = ctypes.c_int
        lib.kpp_rht_inverse.argtypes = [i64, vp, vp, vp, i32, vp]
        lib.kpp_rht_inverse.restype = ctypes.c_int
        i64p = ctypes.POINTER(i64)
        lib.kpp_memo_sequence.argtypes = [ctypes.c_uint64, ctypes.c_uint32, i32, i64, i64, i32, i64, i64, i64, i64p,
                                          i64p, i64, i64p]
        lib.kpp_memo_sequence.restype = ctypes.c_int
        lib.kpp_state_create.argtypes = [i64, i64, i32, i32, ctypes.POINTER(vp)]
        lib.kpp_state_create.restype = ctypes.c_int
        lib.kpp_state_destroy.argtypes = [vp]
        lib.kpp_state_destroy.restype = None
        lib.kpp_state_step.argtypes = [vp]
        lib.kpp_state_step.restype = i64
        lib.kpp_state_bytes.argtypes = [vp]
        lib.kpp_state_bytes.restype = ctypes.c_size_t
        lib.kpp_state_save.argtypes = [vp, vp, vp, ctypes.c_size_t, vp]
        lib.kpp_state_save.restype = ctypes.c_int
        lib.kpp_state_load.argtypes = [vp, vp, vp, ctypes.c_size_t, vp]
        lib.kpp_state_load.restype = ctypes.c_int
        lib.kpp_tune_block_size.argtypes = [i32, ctypes.POINTER(Matrix), ctypes.POINTER(vp), i32,
                                             ctypes.POINTER(i32), i32, ctypes.POINTER(Params), i32,
                                             ctypes.POINTER(i32), ctypes.POINTER(dbl), vp]
        lib.kpp_tune_block_size.restype = ctypes.c_int
        lib.kpp_solve_memo.argtypes = [ctypes.POINTER(Matrix), vp, vp, i32, i32, ctypes.POINTER(Params),
                                       ctypes.POINTER(Report), ctypes.POINTER(i64), vp]
        lib.kpp_solve_memo.restype = ctypes.c_int
        lib.kpp_factor_lsqr.argtypes = [ctypes.POINTER(Matrix), vp, dbl, i64, ctypes.POINTER(i64), vp,
                                        ctypes.POINTER(vp), vp]
        lib.kpp_factor_lsqr.restype = ctypes.c_int
        lib.kpp_proj_lsqr.argtypes = [ctypes.POINTER(Matrix), vp, vp, i64, vp, i32, vp, vp]
        lib.kpp_proj_lsqr.restype = ctypes.c_int
        lib.kpp_solve_lsqr.argtypes = [ctypes.POINTER(Matrix), vp, vp, vp, vp, i32, ctypes.POINTER(Params),
                                       ctypes.POINTER(Report), vp]
        lib.kpp_solve_lsqr.restype = ctypes.c_int
        lib.kpp_cg.argtypes = [ctypes.POINTER(Matrix), vp, vp, dbl, i64, ctypes.POINTER(Report), vp]
        lib.kpp_cg.restype = ctypes.c_int
        lib.kpp_gmres.argtypes = [ctypes.POINTER(Matrix), vp, vp, i32, dbl, i64, ctypes.POINTER(Report), vp]
        lib.kpp_gmres.restype = ctypes.c_int
        for name in ("kpp_solve_resume", "cdpp_solve_resume"):
            getattr(lib, name).argtypes = [ctypes.POINTER(Matrix), vp, vp, vp, vp, ctypes.POINTER(Params), vp,
                                           ctypes.POINTER(Report), vp]
            getattr(lib, name).restype = ctypes.c_int
        for name in ("kpp_set_kernel_variant", "cdpp_solve_noalloc", "kpp_sample_blocks", "kpp_partition", "kpp_factor_blocks", "kpp_factors_get_block", "kpp_solve", "cdpp_solve",
                     "kpp_solve_host", "kpp_rel_residual", "kpp_solve_batched"):
            getattr(lib, name).restype = ctypes.c_int
        lib.kpp_plan_create.argtypes = [i32, ctypes.POINTER(Matrix), ctypes.POINTER(vp), ctypes.POINTER(vp), i32,
                                        vp, ctypes.POINTER(vp), ctypes.POINTER(Params), i32, vp, ctypes.POINTER(vp)]
        lib.kpp_plan_launch.argtypes = [vp, vp]
        lib.kpp_plan_report.argtypes = [vp, ctypes.POINTER(Report), vp]
        lib.kpp_plan_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)]
        lib.kpp_plan_destroy.argtypes = [vp]
        lib.kpp_plan_destroy.restype = None
        lib.kpp_tune_cache_size.restype = i64
        lib.kpp_launch_count.restype = ctypes.c_uint64
        lib.kpp_device_alloc_count.restype = ctypes.c_uint64
        lib.kpp_device_cache_bytes.argtypes = []
        lib.kpp_device_cache_bytes.restype = ctypes.c_size_t
        lib.kpp_device_cache_trim.argtypes = []
        lib.kpp_device_cache_trim.restype = ctypes.c_int
        lib.kpp_tune_cache_clear.restype = None
        lib.kpp_tune_cache_save.argtypes = [ctypes.c_char_p]
        lib.kpp_tune_cache_load.argtypes = [ctypes.c_char_p]
        for name in ("kpp_plan_create", "kpp_plan_launch", "kpp_plan_report", "kpp_plan_info", "kpp_tune_cache_save",
                     "kpp_tune_cache_load"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def last_error() -> str:
    return load().kpp_last_error().decode()


def _check(rc: int, allow=()):
    if rc != OK and rc not in allow:
        raise KppError(rc, last_error())
    return rc


# ---------------------------------------------------------------------------------------------
# torch <-> C structs
# ---------------------------------------------------------------------------------------------

def _dtype_code(t) -> int:
    import torch
    m = {torch.float64: KPP_F64, torch.float32: KPP_F32, torch.bfloat16: KPP_BF16}
    if t.dtype not in m:
        raise TypeError(f"unsupported matrix dtype {t.dtype}")
    return m[t.dtype]


def matrix(A) -> Matrix:
    """Describe a 2-D torch tensor (row-major, unit column stride) as a kpp_matrix."""
    if A.dim() != 2 or A.stride(1) != 1:
        raise ValueError("A must be a 2-D row-major tensor with unit column stride")
    return Matrix(ctypes.c_void_p(A.data_ptr()), _dtype_code(A), 0, A.shape[0], A.shape[1], A.stride(0))


def host_matrix(A) -> Matrix:
    """Describe a C-contiguous numpy array (float64 / float32, or uint16 holding bf16 bits)."""
    import numpy as np
    codes = {np.dtype(np.float64): KPP_F64, np.dtype(np.float32): KPP_F32, np.dtype(np.uint16): KPP_BF16}
    if A.ndim != 2 or not A.flags.c_contiguous or A.dtype not in codes:
        raise ValueError("host matrix must be a C-contiguous 2-D float64/float32/uint16(bf16) array")
    return Matrix(ctypes.c_void_p(A.ctypes.data), codes[A.dtype], 0, A.shape[0], A.shape[1], A.shape[1])


def _stream_ptr(stream) -> ctypes.c_void_p:
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def params(**kw) -> Params:
    """kpp_params_default() with fields overridden (use ``lam`` for lambda)."""
    p = load().kpp_params_default()
    for k, v in kw.items():
        if k in ("lam", "lambda_"):
            p.lambda_ = float(v)
        elif k == "eta" and v is None:
            p.eta = math.nan
        else:
            if not hasattr(p, k):
                raise AttributeError(k)
            setattr(p, k, v)
    return p


# ---------------------------------------------------------------------------------------------
# Handles
# ---------------------------------------------------------------------------------------------

class Partition:
    """Fixed contiguous row partition into blocks of s rows (kpp_partition)."""

    def __init__(self, rows: int, s: int):
        self._lib = load()
        h = ctypes.c_void_p()
        _check(self._lib.kpp_partition(rows, s, ctypes.byref(h)))
        self.handle, self.rows, self.s = h, rows, s

    @property
    def nb(self) -> int:
        return int(self._lib.kpp_partition_blocks(self.handle))

    def __del__(self):
        if getattr(self, "handle", None):
            self._lib.kpp_partition_destroy(self.handle)
            self.handle = None


class Factors:
    """Memoised per-block factors (kpp_factor_blocks).  mode 0: K++ Gram, 1: CD++ principal block."""

    def __init__(self, A, P: Partition, lam: float, mode: int, stream=None, allow_not_spd: bool = False):
        self._lib = load()
        self._A = A  # keep the matrix alive while the factors are
        h = ctypes.c_void_p()
        m = matrix(A)
        rc = self._lib.kpp_factor_blocks(ctypes.byref(m), P.handle, float(lam), int(mode), ctypes.byref(h),
                                         _stream_ptr(stream))
        self.handle = h if h.value else None
        self.status = rc
        _check(rc, allow=(ERR_NOT_SPD,) if allow_not_spd else ())
        self.lam, self.mode, self.P = lam, mode, P

    @property
    def bad_block(self) -> int:
        return int(self._lib.kpp_factors_bad_block(self.handle))

    @property
    def fp64_blocks(self) -> int:
        """Blocks whose Cholesky ran in FP64 (all for FP64 storage; the ill-conditioned ones otherwise)."""
        return int(self._lib.kpp_factors_fp64_blocks(self.handle))

    def stage_ms(self) -> dict:
        """Device time (ms) of the factor phase's stages: Grams (or principal blocks), Cholesky,
        inverses, W memo."""
        out = (ctypes.c_double * 4)()
        _check(self._lib.kpp_factors_stage_ms(self.handle, out))
        return dict(zip(("gram", "cholesky", "inverse", "wmemo"), list(out)))

    def memo(self, row0: int, nrows: int, cols: int):
        """Rows row0 .. row0+nrows-1 of the FP32 memo W (W_j = G_j^-1 A_Sj) as a numpy array."""
        import numpy as np
        out = np.zeros((nrows, cols), dtype=np.float32)
        _check(self._lib.kpp_factors_get_memo(self.handle, int(row0), int(nrows),
                                              out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return out

    def block(self, j: int):
        """FP64 lower Cholesky factor of block j as a numpy array."""
        import numpy as np
        ln = min(self.P.s, self.P.rows - j * self.P.s)
        out = np.zeros((ln, ln))
        _check(self._lib.kpp_factors_get_block(self.handle, j, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    def __del__(self):
        if getattr(self, "handle", None):
            self._lib.kpp_factors_destroy(self.handle)
            self.handle = None


def _report_or_raise(rc: int, rep: Report, allow_no_conv: bool) -> Report:
    allow = (ERR_NO_CONVERGENCE,) if allow_no_conv else ()
    _check(rc, allow=allow)
    return rep


def kpp_solve(A, b, x, P: Partition, F: Factors, prm: Params, stream=None, allow_no_conv: bool = False) -> Report:
    """Kaczmarz++ on device tensors; x (float64, cols) holds x0 and receives the result."""
    rep = Report()
    m = matrix(A)
    rc = load().kpp_solve(ctypes.byref(m), ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()), P.handle,
                          F.handle, ctypes.byref(prm), ctypes.byref(rep), _stream_ptr(stream))
    return _report_or_raise(rc, rep, allow_no_conv)


def cdpp_solve(A, b, x, P: Partition, F: Factors, prm: Params, stream=None, allow_no_conv: bool = False) -> Report:
    """CD++ on device tensors (A symmetric n x n); x holds x0 and receives the result."""
    rep = Report()
    m = matrix(A)
    rc = load().cdpp_solve(ctypes.byref(m), ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()), P.handle,
                           F.handle, ctypes.byref(prm), ctypes.byref(rep), _stream_ptr(stream))
    return _report_or_raise(rc, rep, allow_no_conv)


def cdpp_solve_noalloc(A, b, x, P: Partition, F: Factors, prm: Params, stream=None,
                       allow_no_conv: bool = False) -> Report:
    """CD++ FP64 through the entry point that allocates no device memory (fixed internal scratch;
    n <= 16384, s <= 256).  For callers that cannot allocate device memory.  It runs the general
    CD++ kernel with cdpp_solve's launch shape, i.e. what cdpp_solve runs after set_kernel_variant(1).
    Calls must not overlap on the GPU."""
    rep = Report()
    m = matrix(A)
    rc = load().cdpp_solve_noalloc(ctypes.byref(m), ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                   P.handle, F.handle, ctypes.byref(prm), ctypes.byref(rep), _stream_ptr(stream))
    return _report_or_raise(rc, rep, allow_no_conv)


def tune_block_size(As: list, Bs: list, candidates: list, prm: Params, cd: bool = False, stream=None):
    """kpp_tune_block_size: (best s, {s: estimated ms to prm.tol}) over the candidate block sizes."""
    n = len(As)
    k = Bs[0].shape[1] if Bs[0].dim() == 2 else 1
    mats = (Matrix * n)(*[matrix(a) for a in As])
    bp = (ctypes.c_void_p * n)(*[b.data_ptr() for b in Bs])
    cand = (ctypes.c_int32 * len(candidates))(*candidates)
    est = (ctypes.c_double * len(candidates))()
    out = ctypes.c_int32()
    _check(load().kpp_tune_block_size(n, mats, bp, k, cand, len(candidates), ctypes.byref(prm), int(cd),
                                      ctypes.byref(out), est, _stream_ptr(stream)))
    return out.value, dict(zip(candidates, list(est)))


def solve_memo(A, b, x, s: int, prm: Params, cd: bool = False, stream=None, allow_no_conv: bool = False):
    """kpp_solve_memo: K++ (cd=False) or CD++ with the online block memoisation; returns (report,
    number of memoised blocks)."""
    rep = Report()
    nb = ctypes.c_int64()
    m = matrix(A)
    rc = load().kpp_solve_memo(ctypes.byref(m), ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()), int(s),
                               int(cd), ctypes.byref(prm), ctypes.byref(rep), ctypes.byref(nb), _stream_ptr(stream))
    return _report_or_raise(rc, rep, allow_no_conv), int(nb.value)


class LsqrFactors(Factors):
    """Sketch preconditioners of the LSQR projection for every block (kpp_factor_lsqr): tau sampled
    columns T (host integers in [0, n')) of the Hadamard transform, signs d (device, n' values)."""

    def __init__(self, A, P: Partition, lam: float, T, d, stream=None, allow_not_spd: bool = False):
        import numpy as np
        self._lib = load()
        self._A, self._d = A, d
        Tv = np.ascontiguousarray(T, dtype=np.int64)
        h = ctypes.c_void_p()
        m = matrix(A)
        rc = self._lib.kpp_factor_lsqr(ctypes.byref(m), P.handle, float(lam), int(len(Tv)),
                                       Tv.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), ctypes.c_void_p(d.data_ptr()),
                                       ctypes.byref(h), _stream_ptr(stream))
        self.handle = h if h.value else None
        self.status = rc
        _check(rc, allow=(ERR_NOT_SPD,) if allow_not_spd else ())
        self.lam, self.mode, self.P = lam, 2, P


def proj_lsqr(A, P: Partition, F: LsqrFactors, j: int, r, t_max: int, w, stream=None) -> None:
    """kpp_proj_lsqr: w (device, cols) from t_max LSQR iterations for block j and residual r (device, s)."""
    m = matrix(A)
    _check(load().kpp_proj_lsqr(ctypes.byref(m), P.handle, F.handle, int(j), ctypes.c_void_p(r.data_ptr()),
                                int(t_max), ctypes.c_void_p(w.data_ptr()), _stream_ptr(stream)))


def solve_lsqr(A, b, x, P: Partition, F: LsqrFactors, t_max: int, prm: Params, stream=None,
               allow_no_conv: bool = False) -> Report:
    """kpp_solve_lsqr: K++ with the sketch-preconditioned LSQR projection; x holds x0 and the result."""
    rep = Report()
    m = matrix(A)
    rc = load().kpp_solve_lsqr(ctypes.byref(m), ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                               P.handle, F.handle, int(t_max), ctypes.byref(prm), ctypes.byref(rep),
                               _stream_ptr(stream))
    return _report_or_raise(rc, rep, allow_no_conv)


def cg(A, b, x, tol: float = 1e-8, max_iters: int = 100000, stream=None, allow_no_conv: bool = False) -> Report:
    """kpp_cg: plain FP64 conjugate gradients on the GPU; x holds x0 and receives the result."""
    rep = Report()
    m = matrix(A)
    rc = load().kpp_cg(ctypes.byref(m), ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()), float(tol),
                       int(max_iters), ctypes.byref(rep), _stream_ptr(stream))
    return _report_or_raise(rc, rep, allow_no_conv)


def gmres(A, b, x, restart: int = 256, tol: float = 1e-8, max_iters: int = 100000, stream=None,
          allow_no_conv: bool = False) -> Report:
    """kpp_gmres: restarted FP64 GMRES on the GPU; x holds x0 and receives the result."""
    rep = Report()
    m = matrix(A)
    rc = load().kpp_gmres(ctypes.byref(m), ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                          int(restart), float(tol), int(max_iters), ctypes.byref(rep), _stream_ptr(stream))
    return _report_or_raise(rc, rep, allow_no_conv)


class State:
    """Solver state between calls (kpp_state_*): momentum, CD++ residuals, per-column window scalars and
    the next step index, in device memory owned by the handle."""

    def __init__(self, rows: int, cols: int, k: int = 1, cd: bool = False):
        self._lib = load()
        h = ctypes.c_void_p()
        _check(self._lib.kpp_state_create(int(rows), int(cols), int(k), int(cd), ctypes.byref(h)))
        self.handle, self.rows, self.cols, self.k, self.cd = h, rows, cols, k, cd

    @property
    def step(self) -> int:
        return int(self._lib.kpp_state_step(self.handle))

    def save(self, x, stream=None) -> bytes:
        """The checkpoint of the state and of x (device FP64, cols x k) as bytes."""
        n = int(self._lib.kpp_state_bytes(self.handle))
        buf = ctypes.create_string_buffer(n)
        _check(self._lib.kpp_state_save(self.handle, ctypes.c_void_p(x.data_ptr()), buf, n, _stream_ptr(stream)))
        return buf.raw

    def load(self, data: bytes, x, stream=None) -> None:
        """Restore a checkpoint made by save() into this state and into x."""
        buf = ctypes.create_string_buffer(data, len(data))
        _check(self._lib.kpp_state_load(self.handle, ctypes.c_void_p(x.data_ptr()), buf, len(data),
                                        _stream_ptr(stream)))

    def __del__(self):
        if getattr(self, "handle", None):
            self._lib.kpp_state_destroy(self.handle)
            self.handle = None


def solve_resume(A, b, x, P: Partition, F: Factors, prm: Params, state: State, cd: bool = False, stream=None,
                 allow_no_conv: bool = True) -> list:
    """kpp_solve_resume / cdpp_solve_resume: prm.max_iters more steps from `state`; one report per column."""
    reps = (Report * state.k)()
    m = matrix(A)
    fn = load().cdpp_solve_resume if cd else load().kpp_solve_resume
    rc = fn(ctypes.byref(m), ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()), P.handle, F.handle,
            ctypes.byref(prm), state.handle, reps, _stream_ptr(stream))
    _check(rc, allow=(ERR_NO_CONVERGENCE,) if allow_no_conv else ())
    return list(reps)


def kpp_solve_batched(As: list, Bs: list, Xs: list, P: Partition, Fs: list, prm: Params, stream=None,
                      allow_no_conv: bool = False, cd: bool = False) -> list:
    """Batched K++ (or CD++ with cd=True): systems i with A_i (rows x cols), B_i (rows x k) and X_i
    (cols x k), FP64 panels."""
    n = len(As)
    k = Bs[0].shape[1] if Bs[0].dim() == 2 else 1
    mats = (Matrix * n)(*[matrix(a) for a in As])
    bp = (ctypes.c_void_p * n)(*[b.data_ptr() for b in Bs])
    xp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in Xs])
    fp = (ctypes.c_void_p * n)(*[f.handle.value for f in Fs])
    reps = (Report * (n * k))()
    fn = load().cdpp_solve_batched if cd else load().kpp_solve_batched
    rc = fn(n, mats, bp, xp, k, P.handle, fp, ctypes.byref(prm), reps, _stream_ptr(stream))
    _check(rc, allow=(ERR_NO_CONVERGENCE,) if allow_no_conv else ())
    return list(reps)


class Plan:
    """A prepared batched solve (kpp_plan_create): systems, scratch and launch shape fixed once.
    launch() enqueues the whole solve with kernels and memsets only, so it can be captured into a
    torch.cuda.CUDAGraph and replayed; report() synchronises and returns nsys * k reports."""

    def __init__(self, As: list, Bs: list, Xs: list, P: Partition, Fs: list, prm: Params, cd: bool = False,
                 stream=None):
        self._lib = load()
        n = len(As)
        self.nsys = n
        self.k = Bs[0].shape[1] if Bs[0].dim() == 2 else 1
        self._keep = (As, Bs, Xs, P, Fs)  # the plan holds their device addresses
        mats = (Matrix * n)(*[matrix(a) for a in As])
        bp = (ctypes.c_void_p * n)(*[b.data_ptr() for b in Bs])
        xp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in Xs])
        fp = (ctypes.c_void_p * n)(*[f.handle.value for f in Fs])
        self.handle = ctypes.c_void_p()
        _check(self._lib.kpp_plan_create(n, mats, bp, xp, self.k, P.handle, fp, ctypes.byref(prm), 1 if cd else 0,
                                         _stream_ptr(stream), ctypes.byref(self.handle)))

    def launch(self, stream=None) -> None:
        _check(self._lib.kpp_plan_launch(self.handle, _stream_ptr(stream)))

    def report(self, stream=None, allow_no_conv: bool = False) -> list:
        reps = (Report * (self.nsys * self.k))()
        rc = self._lib.kpp_plan_report(self.handle, reps, _stream_ptr(stream))
        _check(rc, allow=(ERR_NO_CONVERGENCE,) if allow_no_conv else ())
        return list(reps)

    def info(self) -> dict:
        kern, grid, var = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(self._lib.kpp_plan_info(self.handle, ctypes.byref(kern), ctypes.byref(grid), ctypes.byref(var)))
        return {"kernel": kern.value, "grid": grid.value, "variant": var.value}

    def close(self) -> None:
        if getattr(self, "handle", None):
            self._lib.kpp_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()


def launch_count() -> int:
    """Kernel launches the library has issued in this process."""
    return int(load().kpp_launch_count())


def device_alloc_count() -> int:
    """Device allocation requests the library has made in this process (cached ones included)."""
    return int(load().kpp_device_alloc_count())


def device_cache_bytes() -> int:
    """kpp_device_cache_bytes: device memory the library holds for reuse on the current device."""
    return int(load().kpp_device_cache_bytes())


def device_cache_trim() -> None:
    """kpp_device_cache_trim: return the library's cached device memory to the driver."""
    _check(load().kpp_device_cache_trim())


def tune_cache_size() -> int:
    return int(load().kpp_tune_cache_size())


def tune_cache_clear() -> None:
    load().kpp_tune_cache_clear()


def tune_cache_save(path: str) -> None:
    _check(load().kpp_tune_cache_save(str(path).encode()))


def tune_cache_load(path: str) -> None:
    _check(load().kpp_tune_cache_load(str(path).encode()))


def solve_host(A_np, b_np, x_np, s: int, mode: int, prm: Params, stream=None) -> Report:
    """End-to-end call on host (numpy) buffers: copies in, factors, solves, copies x back."""
    import numpy as np
    m = host_matrix(A_np)
    assert b_np.dtype == np.float64 and x_np.dtype == np.float64 and x_np.flags.c_contiguous
    rep = Report()
    rc = load().kpp_solve_host(ctypes.byref(m), ctypes.c_void_p(b_np.ctypes.data), ctypes.c_void_p(x_np.ctypes.data),
                               int(s), int(mode), ctypes.byref(prm), ctypes.byref(rep), _stream_ptr(stream))
    _check(rc, allow=(ERR_NO_CONVERGENCE,))
    return rep


def rel_residual(A, b, x, stream=None) -> float:
    """|A x - b| / |b| with FP64 accumulation, on the device."""
    out = ctypes.c_double()
    m = matrix(A)
    _check(load().kpp_rel_residual(ctypes.byref(m), ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                   ctypes.byref(out), _stream_ptr(stream)))
    return out.value


def sample_blocks(seed: int, sys_id: int, t0: int, count: int, nb: int, stream=None):
    """Device-drawn block indices for steps t0..t0+count-1 (int32 CUDA tensor)."""
    import torch
    out = torch.empty(count, dtype=torch.int32, device="cuda")
    _check(load().kpp_sample_blocks(seed, sys_id, t0, count, nb, ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


def block_gram(A, s: int, lam: float, engine: int = 0, stream=None):
    """Lower triangles of the block Grams A_S A_S^T + lam I (FP64, (nb, s, s) packed per block) and the
    engine used (1 CUDA cores FP64-accumulate, 2 tensor cores FP32-accumulate)."""
    import torch
    nb = -(-A.shape[0] // s)
    G = torch.zeros(nb * s * s, dtype=torch.float64, device=A.device)
    used = ctypes.c_int32(-1)
    m = matrix(A)
    _check(load().kpp_block_gram(ctypes.byref(m), int(s), float(lam), int(engine), ctypes.c_void_p(G.data_ptr()),
                                 ctypes.byref(used), _stream_ptr(stream)))
    return G, used.value


def memo_sequence(seed: int, sys_id: int, cd: bool, rows: int, cols: int, s: int, t0: int, count: int, nb0: int = 0):
    """The online memo's block sequence for steps t0 .. t0+count-1 (kpp_memo_sequence): (memo index per
    step, the new blocks' row subsets (new x s), number of memoised blocks after the window)."""
    import numpy as np
    blocks = np.empty(max(count, 1), dtype=np.int64)
    subsets = np.empty((max(count, 1), s), dtype=np.int64)
    nb = ctypes.c_int64()
    p = ctypes.POINTER(ctypes.c_int64)
    _check(load().kpp_memo_sequence(seed, sys_id, int(cd), rows, cols, s, t0, count, nb0,
                                    blocks.ctypes.data_as(p), subsets.ctypes.data_as(p), count, ctypes.byref(nb)))
    return blocks[:count], subsets[: nb.value - nb0], nb.value


def rht_forward(d, A, b=None, stream=None):
    """(Q A Q^T, Q b) with Q = H_n diag(d) / sqrt(n) (kpp_rht_forward): d FP64 signs, A FP64 n x n, b a
    vector or n x k panel (FP64) or None.  Returns new device tensors."""
    import torch
    n = A.shape[0]
    Abar = torch.empty((n, n), dtype=torch.float64, device=A.device)
    m = matrix(A)
    if b is None:
        bb, bbar, k = None, None, 0
    else:
        bb = b.reshape(n, -1).contiguous()
        bbar = torch.empty_like(bb)
        k = bb.shape[1]
    vp = ctypes.c_void_p
    _check(load().kpp_rht_forward(n, vp(d.data_ptr()), ctypes.byref(m), vp(Abar.data_ptr()),
                                  vp(bb.data_ptr() if bb is not None else 0), vp(bbar.data_ptr() if bbar is not None else 0),
                                  k, _stream_ptr(stream)))
    return Abar, (None if b is None else bbar.reshape(b.shape))


def rht_inverse(d, xbar, stream=None):
    """x = Q^T xbar = diag(d) H_n xbar / sqrt(n) (kpp_rht_inverse) for a vector or n x k panel."""
    n = xbar.shape[0]
    xb = xbar.reshape(n, -1).contiguous()
    x = xb.new_empty(xb.shape)
    _check(load().kpp_rht_inverse(n, ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(xb.data_ptr()),
                                  ctypes.c_void_p(x.data_ptr()), xb.shape[1], _stream_ptr(stream)))
    return x.reshape(xbar.shape)


class Server:
    """Continuous-batching solve server (kpp_server_*): admission by a device-memory budget, memoised
    factors kept resident per registered matrix, and a device-resident request loop whose slots
    (max_concurrent of them, grid_per_solve CTAs each) claim and run the queued jobs."""

    def __init__(self, hbm_budget_bytes: int, max_concurrent: int = 8, grid_per_solve: int = 0):
        self._lib = load()
        h = ctypes.c_void_p()
        _check(self._lib.kpp_server_create(int(hbm_budget_bytes), int(max_concurrent), int(grid_per_solve),
                                           ctypes.byref(h)))
        self.handle = h
        self._mats = []

    def add_matrix(self, A, s: int, lam: float, mode: int) -> int:
        mid = ctypes.c_int32()
        m = matrix(A)
        _check(self._lib.kpp_server_add_matrix(self.handle, ctypes.byref(m), int(s), float(lam), int(mode),
                                               ctypes.byref(mid)))
        self._mats.append(A)  # the device matrix must outlive the server
        return mid.value

    def submit(self, matrix_id: int, B, prm: Params) -> int:
        import numpy as np
        B = np.ascontiguousarray(B, dtype=np.float64)
        k = 1 if B.ndim == 1 else B.shape[1]
        rid = ctypes.c_int64()
        rc = self._lib.kpp_server_submit(self.handle, int(matrix_id), ctypes.c_void_p(B.ctypes.data), k,
                                         ctypes.byref(prm), ctypes.byref(rid))
        _check(rc, allow=(ERR_BUDGET,))
        return rid.value

    def poll(self, request_id: int, cols: int, k: int):
        """(done, status, X (cols x k) or None, reports or None)."""
        import numpy as np
        X = np.zeros((cols, k))
        reps = (Report * k)()
        done = ctypes.c_int32()
        rc = self._lib.kpp_server_poll(self.handle, int(request_id), ctypes.c_void_p(X.ctypes.data), reps,
                                       ctypes.byref(done))
        if not done.value:
            return False, None, None, None
        return True, rc, X, list(reps)

    def wait_all(self, timeout_s: float = 600.0):
        _check(self._lib.kpp_server_wait_all(self.handle, float(timeout_s)))

    def stats(self) -> dict:
        st = ServingStats()
        _check(self._lib.kpp_server_stats(self.handle, ctypes.byref(st)))
        return st.as_dict()

    def reset_stats(self) -> None:
        _check(self._lib.kpp_server_reset_stats(self.handle))

    def close(self):
        if getattr(self, "handle", None):
            self._lib.kpp_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()


def set_kernel_variant(v: int) -> None:
    """1: general kernel everywhere; 2: small-block kernel where the shape allows it; 3 (default): as 2,
    and the dataflow kernel for CD++ where the shape allows it."""
    _check(load().kpp_set_kernel_variant(int(v)))


def set_wait_test(wait_ns: int = 0, hold_cta: int = -1) -> None:
    """Test hook: the device wait limit of later launches (0: the default 2 s) and the CTA that the
    general kernel holds back from its first group barrier (-1: none), so that a bounded wait runs out."""
    _check(load().kpp_set_wait_test(int(wait_ns), int(hold_cta)))


def build_info() -> str:
    return load().kpp_build_info().decode()
