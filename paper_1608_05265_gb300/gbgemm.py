"""Thin ctypes binding over libgbgemm.so (argument marshalling only).

Every function has the name and argument order of its C counterpart in
``include/gbgemm.h``; torch tensors are passed by ``data_ptr()`` and the
stream as ``torch.cuda.Stream.cuda_stream``.  Matrices are column-major: a
column-major m x n matrix with leading dimension ld is a torch tensor whose
storage holds n columns of ld floats (for example ``t.T`` of a row-major
(n, ld) tensor).  There is no fallback: if the library is missing or cannot
be loaded, ``lib()`` raises.
"""

from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libgbgemm.so")

OK = 0
ERR_NOT_INITIALIZED = -100
ERR_ALLOC = -101
ERR_CUDA = -102
ERR_UNSUPPORTED_DEVICE = -103
ERR_DEVICE_TIMEOUT = -104
ERR_BAD_PLAN = -105
ERR_INVALID_VALUE = -106
ERR_SCRATCH_LIMIT = -107
NOALLOC_SCRATCH_BYTES = 64 * 1024 * 1024
MLP_PARAMS = 5126
SCHED_MLP_PARAMS = 7271
NUM_SCHEDULES = 39

PATH_AUTO = 0
PATH_SIMT = 1
PATH_SPLIT_BF16 = 2

CFG_SIMT_128x128 = 0
CFG_SIMT_64x64 = 1
CFG_SIMT_128x64 = 2
CFG_SPLIT_BN64 = 3
CFG_SPLIT_BN128 = 4
CFG_SPLIT_BN256 = 5
NUM_CONFIGS = 6

CONFIG_PREDICTED = 0
CONFIG_TUNED = 1
CONFIG_DEFAULT = 2


class Problem(ctypes.Structure):
    """gbgemm_problem (include/gbgemm.h)."""
    _fields_ = [("transa", ctypes.c_char), ("transb", ctypes.c_char),
                ("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int64),
                ("alpha", ctypes.c_float), ("beta", ctypes.c_float),
                ("A", ctypes.c_void_p), ("lda", ctypes.c_int64),
                ("B", ctypes.c_void_p), ("ldb", ctypes.c_int64),
                ("C", ctypes.c_void_p), ("ldc", ctypes.c_int64)]

#: Symbols exported by libgbgemm.so, as declared in include/gbgemm.h.
EXPORTS = [
    "gbgemm_create", "gbgemm_destroy", "gbgemm_set_stream", "gbgemm_set_path", "gbgemm_last_path",
    "gbgemm_reserve_workspace", "gbgemm_split_workspace_bytes", "gbgemm_sgemm", "gbgemm_sgemm_strided_batched",
    "gbgemm_sgemv", "gbgemm_sgetrf", "gbgemm_sgetrs",
    "gbgemm_get_device_status", "gbgemm_debug_expire_wait",
    "gbgemm_status_string", "gbgemm_panel_bytes", "gbgemm_split_pack", "gbgemm_profile_begin",
    "gbgemm_profile_end", "gbgemm_sgemm_split_noalloc", "gbgemm_grouped_plan_create",
    "gbgemm_grouped_plan_create_with_configs", "gbgemm_grouped_plan_run", "gbgemm_grouped_plan_configs",
    "gbgemm_grouped_plan_stats", "gbgemm_grouped_plan_destroy", "gbgemm_autotune", "gbgemm_tuning_save",
    "gbgemm_tuning_load", "gbgemm_tuning_clear", "gbgemm_set_tuning", "gbgemm_predictor_set",
    "gbgemm_predictor_get", "gbgemm_predictor_features", "gbgemm_predictor_predict",
    "gbgemm_predictor_loss_grad", "gbgemm_predictor_train", "gbgemm_check_error",
    "gbgemm_schedule_info", "gbgemm_schedule_legal", "gbgemm_schedule_default", "gbgemm_autotune_schedules",
    "gbgemm_last_schedule", "gbgemm_set_schedule", "gbgemm_predictor_select",
]

_lock = threading.Lock()
_lib = None


class GbgemmError(RuntimeError):
    def __init__(self, fn: str, status: int):
        super().__init__(f"{fn} returned {status} ({status_string(status)})")
        self.status = status


def lib():
    """Load libgbgemm.so (built by paper_1608_05265_gb300.build); raise if absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: run paper_1608_05265_gb300.build.build() first")
            L = ctypes.CDLL(LIB_PATH)
            vp, i64, f32, c = ctypes.c_void_p, ctypes.c_int64, ctypes.c_float, ctypes.c_char
            L.gbgemm_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int]
            L.gbgemm_destroy.argtypes = [vp]
            L.gbgemm_set_stream.argtypes = [vp, vp]
            L.gbgemm_set_path.argtypes = [vp, ctypes.c_int]
            L.gbgemm_last_path.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
            L.gbgemm_reserve_workspace.argtypes = [vp, ctypes.c_size_t]
            L.gbgemm_split_workspace_bytes.argtypes = [i64, i64, i64]
            L.gbgemm_split_workspace_bytes.restype = ctypes.c_size_t
            L.gbgemm_sgemm.argtypes = [vp, c, c, i64, i64, i64, f32, vp, i64, vp, i64, f32, vp, i64]
            L.gbgemm_sgemm_strided_batched.argtypes = [vp, c, c, i64, i64, i64, f32, vp, i64, i64, vp, i64, i64, f32,
                                                       vp, i64, i64, i64]
            L.gbgemm_sgemv.argtypes = [vp, c, i64, i64, f32, vp, i64, vp, i64, f32, vp, i64]
            L.gbgemm_sgetrf.argtypes = [vp, i64, vp, i64, vp, vp, ctypes.c_int]
            L.gbgemm_sgetrs.argtypes = [vp, i64, i64, vp, i64, vp, vp, i64]
            L.gbgemm_get_device_status.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
            L.gbgemm_debug_expire_wait.argtypes = [vp, ctypes.c_uint64]
            L.gbgemm_status_string.argtypes = [ctypes.c_int]
            L.gbgemm_status_string.restype = ctypes.c_char_p
            L.gbgemm_panel_bytes.argtypes = [i64, i64]
            L.gbgemm_panel_bytes.restype = ctypes.c_size_t
            L.gbgemm_split_pack.argtypes = [vp, c, c, i64, i64, vp, i64, vp, vp, vp]
            L.gbgemm_sgemm_split_noalloc.argtypes = [vp, c, c, i64, i64, i64, f32, vp, i64, vp, i64, f32, vp, i64,
                                                     vp]
            PP = ctypes.POINTER(Problem)
            L.gbgemm_grouped_plan_create.argtypes = [vp, PP, i64, ctypes.c_int, ctypes.POINTER(vp),
                                                     ctypes.POINTER(i64)]
            L.gbgemm_grouped_plan_create_with_configs.argtypes = [vp, PP, i64, ctypes.POINTER(ctypes.c_int),
                                                                  ctypes.POINTER(vp), ctypes.POINTER(i64)]
            L.gbgemm_grouped_plan_run.argtypes = [vp, vp]
            L.gbgemm_grouped_plan_configs.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
            L.gbgemm_grouped_plan_stats.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64),
                                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                                    ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_size_t)]
            L.gbgemm_grouped_plan_destroy.argtypes = [vp]
            fp = ctypes.POINTER(ctypes.c_float)
            ip = ctypes.POINTER(ctypes.c_int)
            L.gbgemm_autotune.argtypes = [vp, PP, ctypes.c_int, fp, fp, ip, ip]
            L.gbgemm_tuning_save.argtypes = [vp, ctypes.c_char_p]
            L.gbgemm_tuning_load.argtypes = [vp, ctypes.c_char_p]
            L.gbgemm_tuning_clear.argtypes = [vp]
            L.gbgemm_set_tuning.argtypes = [vp, ctypes.c_int]
            L.gbgemm_predictor_set.argtypes = [vp, vp]
            L.gbgemm_predictor_get.argtypes = [vp, vp]
            L.gbgemm_predictor_features.argtypes = [PP, fp]
            L.gbgemm_predictor_predict.argtypes = [vp, vp, vp, i64, vp, vp]
            L.gbgemm_predictor_loss_grad.argtypes = [vp, vp, vp, vp, i64, fp, vp]
            L.gbgemm_predictor_train.argtypes = [vp, vp, vp, vp, i64, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                                 ctypes.c_uint64, fp]
            L.gbgemm_check_error.argtypes = [vp, c, c, i64, i64, i64, f32, vp, i64, vp, i64, f32, vp, vp, i64, i64,
                                             i64, i64, i64, ctypes.POINTER(ctypes.c_double)]
            L.gbgemm_schedule_info.argtypes = [ctypes.c_int, ip, ip, ip, ip, ip]
            L.gbgemm_schedule_legal.argtypes = [vp, PP, ctypes.c_int, ip]
            L.gbgemm_schedule_default.argtypes = [vp, PP, ip]
            L.gbgemm_autotune_schedules.argtypes = [vp, PP, ctypes.c_int, fp, ip]
            L.gbgemm_last_schedule.argtypes = [vp, ip]
            L.gbgemm_set_schedule.argtypes = [vp, ctypes.c_int]
            L.gbgemm_predictor_select.argtypes = [vp, ctypes.c_int]
            L.gbgemm_profile_begin.argtypes = [vp]
            L.gbgemm_profile_end.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64),
                                             ctypes.POINTER(i64)]
            for name in ("gbgemm_create", "gbgemm_destroy", "gbgemm_set_stream", "gbgemm_set_path",
                         "gbgemm_last_path", "gbgemm_reserve_workspace", "gbgemm_sgemm",
                         "gbgemm_sgemm_strided_batched", "gbgemm_sgemv", "gbgemm_sgetrf", "gbgemm_sgetrs",
                         "gbgemm_get_device_status", "gbgemm_debug_expire_wait", "gbgemm_split_pack",
                         "gbgemm_profile_begin",
                         "gbgemm_profile_end", "gbgemm_sgemm_split_noalloc", "gbgemm_grouped_plan_create",
                         "gbgemm_grouped_plan_create_with_configs", "gbgemm_grouped_plan_run",
                         "gbgemm_grouped_plan_configs", "gbgemm_grouped_plan_stats",
                         "gbgemm_grouped_plan_destroy", "gbgemm_autotune", "gbgemm_tuning_save",
                         "gbgemm_tuning_load", "gbgemm_tuning_clear", "gbgemm_set_tuning", "gbgemm_predictor_set",
                         "gbgemm_predictor_get", "gbgemm_predictor_features", "gbgemm_predictor_predict",
                         "gbgemm_predictor_loss_grad", "gbgemm_predictor_train", "gbgemm_check_error",
                         "gbgemm_schedule_info", "gbgemm_schedule_legal", "gbgemm_schedule_default",
                         "gbgemm_autotune_schedules", "gbgemm_last_schedule", "gbgemm_set_schedule",
                         "gbgemm_predictor_select"):
                getattr(L, name).restype = ctypes.c_int
            _lib = L
    return _lib


def status_string(s: int) -> str:
    try:
        return lib().gbgemm_status_string(int(s)).decode()
    except Exception:  # library not loadable: plain number
        return str(s)


def _check(fn: str, rc: int) -> int:
    if rc != OK:
        raise GbgemmError(fn, rc)
    return rc


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else stream


class Handle:
    """Owns a gbgemm_handle; every method forwards to the C function of the same name."""

    def __init__(self, device: int = 0):
        h = ctypes.c_void_p()
        _check("gbgemm_create", lib().gbgemm_create(ctypes.byref(h), int(device)))
        self._h = h
        self.device = device

    @property
    def ptr(self):
        return self._h

    def close(self):
        if self._h is not None and self._h.value:
            lib().gbgemm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream=None):
        _check("gbgemm_set_stream", lib().gbgemm_set_stream(self._h, _stream_ptr(stream)))

    def set_path(self, path: int):
        _check("gbgemm_set_path", lib().gbgemm_set_path(self._h, int(path)))

    def last_path(self) -> int:
        v = ctypes.c_int()
        _check("gbgemm_last_path", lib().gbgemm_last_path(self._h, ctypes.byref(v)))
        return v.value

    def reserve_workspace(self, nbytes: int):
        _check("gbgemm_reserve_workspace", lib().gbgemm_reserve_workspace(self._h, int(nbytes)))

    def sgemm(self, transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, check=True) -> int:
        rc = lib().gbgemm_sgemm(self._h, transa.encode() if isinstance(transa, str) else transa,
                                transb.encode() if isinstance(transb, str) else transb,
                                int(m), int(n), int(k), float(alpha), _ptr(A), int(lda), _ptr(B), int(ldb),
                                float(beta), _ptr(C), int(ldc))
        if check:
            _check("gbgemm_sgemm", rc)
        return rc

    def sgemm_strided_batched(self, transa, transb, m, n, k, alpha, A, lda, stride_a, B, ldb, stride_b, beta,
                              C, ldc, stride_c, batch, check=True) -> int:
        rc = lib().gbgemm_sgemm_strided_batched(
            self._h, transa.encode() if isinstance(transa, str) else transa,
            transb.encode() if isinstance(transb, str) else transb, int(m), int(n), int(k), float(alpha), _ptr(A),
            int(lda), int(stride_a), _ptr(B), int(ldb), int(stride_b), float(beta), _ptr(C), int(ldc), int(stride_c),
            int(batch))
        if check:
            _check("gbgemm_sgemm_strided_batched", rc)
        return rc

    def sgemv(self, trans, m, n, alpha, A, lda, x, incx, beta, y, incy, check=True) -> int:
        rc = lib().gbgemm_sgemv(self._h, trans.encode() if isinstance(trans, str) else trans, int(m), int(n),
                                float(alpha), _ptr(A), int(lda), _ptr(x), int(incx), float(beta), _ptr(y), int(incy))
        if check:
            _check("gbgemm_sgemv", rc)
        return rc

    def sgetrf(self, n, A, lda, ipiv, info, nb=0, check=True) -> int:
        """P A = L U in place (ipiv: n int32, info: one int32, both on the device)."""
        rc = lib().gbgemm_sgetrf(self._h, int(n), _ptr(A), int(lda), _ptr(ipiv), _ptr(info), int(nb))
        if check:
            _check("gbgemm_sgetrf", rc)
        return rc

    def sgetrs(self, n, nrhs, LU, lda, ipiv, B, ldb, check=True) -> int:
        """B := A^-1 B from the factors of sgetrf."""
        rc = lib().gbgemm_sgetrs(self._h, int(n), int(nrhs), _ptr(LU), int(lda), _ptr(ipiv), _ptr(B), int(ldb))
        if check:
            _check("gbgemm_sgetrs", rc)
        return rc

    def get_device_status(self) -> int:
        v = ctypes.c_int()
        _check("gbgemm_get_device_status", lib().gbgemm_get_device_status(self._h, ctypes.byref(v)))
        return v.value

    def debug_expire_wait(self, timeout_ns: int):
        """Queue a bounded wait that nothing completes (failure-detection test)."""
        _check("gbgemm_debug_expire_wait", lib().gbgemm_debug_expire_wait(self._h, int(timeout_ns)))

    def profile_begin(self):
        _check("gbgemm_profile_begin", lib().gbgemm_profile_begin(self._h))

    def profile_end(self):
        """(summed GEMM kernel ms, GEMM launches, kernels launched) since profile_begin."""
        ms, g, k = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
        _check("gbgemm_profile_end", lib().gbgemm_profile_end(self._h, ctypes.byref(ms), ctypes.byref(g),
                                                              ctypes.byref(k)))
        return ms.value, g.value, k.value

    def autotune(self, prob: "Problem", reps: int = 3):
        """(latency_us[6], cost_us[6], best_by_latency, best_by_cost); -1 marks illegal configurations."""
        lat = (ctypes.c_float * NUM_CONFIGS)()
        cost = (ctypes.c_float * NUM_CONFIGS)()
        bl, bc = ctypes.c_int(), ctypes.c_int()
        _check("gbgemm_autotune", lib().gbgemm_autotune(self._h, ctypes.byref(prob), int(reps), lat, cost,
                                                        ctypes.byref(bl), ctypes.byref(bc)))
        return list(lat), list(cost), bl.value, bc.value

    def tuning_save(self, path: str):
        _check("gbgemm_tuning_save", lib().gbgemm_tuning_save(self._h, path.encode()))

    def tuning_load(self, path: str):
        _check("gbgemm_tuning_load", lib().gbgemm_tuning_load(self._h, path.encode()))

    def tuning_clear(self):
        _check("gbgemm_tuning_clear", lib().gbgemm_tuning_clear(self._h))

    def set_tuning(self, mode: int):
        _check("gbgemm_set_tuning", lib().gbgemm_set_tuning(self._h, int(mode)))

    def predictor_select(self, which: int):
        """0: the grouped configurations' network, 1: the single-call schedules' network."""
        _check("gbgemm_predictor_select", lib().gbgemm_predictor_select(self._h, int(which)))
        self._pred_sel = int(which)

    def _pred_params(self) -> int:
        return SCHED_MLP_PARAMS if getattr(self, "_pred_sel", 0) == 1 else MLP_PARAMS

    def predictor_set(self, params):
        import numpy as np
        arr = np.ascontiguousarray(params, dtype=np.float32)
        assert arr.size == self._pred_params()
        _check("gbgemm_predictor_set", lib().gbgemm_predictor_set(self._h, arr.ctypes.data))

    def predictor_get(self):
        import numpy as np
        arr = np.zeros(self._pred_params(), dtype=np.float32)
        _check("gbgemm_predictor_get", lib().gbgemm_predictor_get(self._h, arr.ctypes.data))
        return arr

    def schedule_legal(self, prob: "Problem", s: int) -> bool:
        v = ctypes.c_int()
        _check("gbgemm_schedule_legal", lib().gbgemm_schedule_legal(self._h, ctypes.byref(prob), int(s),
                                                                    ctypes.byref(v)))
        return bool(v.value)

    def schedule_default(self, prob: "Problem") -> int:
        v = ctypes.c_int()
        _check("gbgemm_schedule_default", lib().gbgemm_schedule_default(self._h, ctypes.byref(prob), ctypes.byref(v)))
        return v.value

    def autotune_schedules(self, prob: "Problem", reps: int = 3):
        """(latency_us[39], best); -1 marks illegal schedules."""
        lat = (ctypes.c_float * NUM_SCHEDULES)()
        b = ctypes.c_int()
        _check("gbgemm_autotune_schedules", lib().gbgemm_autotune_schedules(self._h, ctypes.byref(prob), int(reps),
                                                                            lat, ctypes.byref(b)))
        return list(lat), b.value

    def set_schedule(self, s: int):
        """Pin single-call schedule s (-1 unpins)."""
        _check("gbgemm_set_schedule", lib().gbgemm_set_schedule(self._h, int(s)))

    def last_schedule(self) -> int:
        v = ctypes.c_int()
        _check("gbgemm_last_schedule", lib().gbgemm_last_schedule(self._h, ctypes.byref(v)))
        return v.value

    def predictor_predict(self, x, legal, scores=None, configs=None):
        """Device tensors: x (n x 8 float32), legal (n uint8); fills scores (n x 6) and configs (n int32)."""
        n = int(x.shape[0])
        _check("gbgemm_predictor_predict", lib().gbgemm_predictor_predict(
            self._h, _ptr(x), _ptr(legal), n, _ptr(scores), _ptr(configs)))

    def predictor_loss_grad(self, x, y, mask, grad) -> float:
        loss = ctypes.c_float()
        _check("gbgemm_predictor_loss_grad", lib().gbgemm_predictor_loss_grad(
            self._h, _ptr(x), _ptr(y), _ptr(mask), int(x.shape[0]), ctypes.byref(loss), _ptr(grad)))
        return loss.value

    def predictor_train(self, x, y, mask, epochs, batch=256, lr=1e-3, seed=0) -> float:
        loss = ctypes.c_float()
        _check("gbgemm_predictor_train", lib().gbgemm_predictor_train(
            self._h, _ptr(x), _ptr(y), _ptr(mask), int(x.shape[0]), int(epochs), int(batch), float(lr),
            int(seed), ctypes.byref(loss)))
        return loss.value

    def check_error(self, transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C_in, C_out, ldc,
                    rows=None, cols=None) -> float:
        """Max FP64 error ratio of C_out over a block (gbgemm_check_error)."""
        i0, i1 = rows if rows is not None else (0, m)
        j0, j1 = cols if cols is not None else (0, n)
        r = ctypes.c_double()
        _check("gbgemm_check_error", lib().gbgemm_check_error(
            self._h, transa.encode(), transb.encode(), int(m), int(n), int(k), float(alpha), _ptr(A), int(lda),
            _ptr(B), int(ldb), float(beta), _ptr(C_in), _ptr(C_out), int(ldc), int(i0), int(i1), int(j0), int(j1),
            ctypes.byref(r)))
        return r.value

    def split_pack(self, which, trans, rows, k, X, ldx, amax_bits, panel, panel2=None) -> int:
        return lib().gbgemm_split_pack(self._h, which.encode(), trans.encode(), int(rows), int(k), _ptr(X), int(ldx),
                                       _ptr(amax_bits), _ptr(panel), _ptr(panel2))


class GroupedPlan:
    """Owns a gbgemm_grouped_plan; methods forward to the C functions of the same name."""

    def __init__(self, handle: "Handle", problems, config_source: int = CONFIG_DEFAULT, configs=None):
        arr = (Problem * max(len(problems), 1))(*problems)
        p = ctypes.c_void_p()
        bad = ctypes.c_int64(-1)
        if configs is not None:
            carr = (ctypes.c_int * max(len(configs), 1))(*configs)
            rc = lib().gbgemm_grouped_plan_create_with_configs(handle.ptr, arr, len(problems), carr, ctypes.byref(p),
                                                               ctypes.byref(bad))
        else:
            rc = lib().gbgemm_grouped_plan_create(handle.ptr, arr, len(problems), int(config_source), ctypes.byref(p),
                                                  ctypes.byref(bad))
        self.bad_index = bad.value
        _check("gbgemm_grouped_plan_create", rc)
        self._p = p
        self.count = len(problems)

    def run(self, stream=None):
        _check("gbgemm_grouped_plan_run", lib().gbgemm_grouped_plan_run(self._p, _stream_ptr(stream)))

    def configs(self):
        arr = (ctypes.c_int * max(self.count, 1))()
        _check("gbgemm_grouped_plan_configs", lib().gbgemm_grouped_plan_configs(self._p, arr))
        return list(arr)[: self.count]

    def stats(self):
        ns, nm = ctypes.c_int64(), ctypes.c_int64()
        fs, fm = ctypes.c_double(), ctypes.c_double()
        kr, db = ctypes.c_int(), ctypes.c_size_t()
        _check("gbgemm_grouped_plan_stats", lib().gbgemm_grouped_plan_stats(
            self._p, ctypes.byref(ns), ctypes.byref(nm), ctypes.byref(fs), ctypes.byref(fm), ctypes.byref(kr),
            ctypes.byref(db)))
        return {"n_split": ns.value, "n_simt": nm.value, "flops_split": fs.value, "flops_simt": fm.value,
                "kernels_per_run": kr.value, "device_bytes": db.value}

    def close(self):
        if getattr(self, "_p", None) is not None and self._p.value:
            lib().gbgemm_grouped_plan_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def create_plan_status(handle, problems, config_source=CONFIG_DEFAULT, configs=None):
    """(status, bad_index) of a plan creation attempt; the plan, if any, is destroyed at once."""
    arr = (Problem * max(len(problems), 1))(*problems)
    p = ctypes.c_void_p()
    bad = ctypes.c_int64(-1)
    if configs is not None:
        carr = (ctypes.c_int * max(len(configs), 1))(*configs)
        rc = lib().gbgemm_grouped_plan_create_with_configs(handle.ptr, arr, len(problems), carr, ctypes.byref(p),
                                                           ctypes.byref(bad))
    else:
        rc = lib().gbgemm_grouped_plan_create(handle.ptr, arr, len(problems), int(config_source), ctypes.byref(p),
                                              ctypes.byref(bad))
    if rc == OK and p.value:
        lib().gbgemm_grouped_plan_destroy(p)
    return rc, bad.value


def problem(transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc) -> Problem:
    """A gbgemm_problem from tensors (or raw device addresses)."""
    return Problem(transa.encode(), transb.encode(), int(m), int(n), int(k), float(alpha), float(beta),
                   _ptr(A), int(lda), _ptr(B), int(ldb), _ptr(C), int(ldc))


def sgemm_split_noalloc(stream, transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, status=None) -> int:
    """gbgemm_sgemm_split_noalloc: the split-path sgemm with no device allocation (returns the status)."""
    return lib().gbgemm_sgemm_split_noalloc(_stream_ptr(stream), transa.encode(), transb.encode(), int(m), int(n),
                                            int(k), float(alpha), _ptr(A), int(lda), _ptr(B), int(ldb), float(beta),
                                            _ptr(C), int(ldc), _ptr(status))


def predictor_features(prob: "Problem"):
    arr = (ctypes.c_float * 8)()
    _check("gbgemm_predictor_features", lib().gbgemm_predictor_features(ctypes.byref(prob), arr))
    return list(arr)


def split_workspace_bytes(m, n, k) -> int:
    return int(lib().gbgemm_split_workspace_bytes(int(m), int(n), int(k)))


def panel_bytes(rows, k) -> int:
    return int(lib().gbgemm_panel_bytes(int(rows), int(k)))


def schedule_info(s: int) -> dict:
    """Decode single-call schedule s (host only): path, tile rows and columns, raster, k-slicing level."""
    v = [ctypes.c_int() for _ in range(5)]
    _check("gbgemm_schedule_info", lib().gbgemm_schedule_info(int(s), *[ctypes.byref(x) for x in v]))
    return {"path": v[0].value, "tile_m": v[1].value, "tile_n": v[2].value, "raster": v[3].value,
            "level": v[4].value}
