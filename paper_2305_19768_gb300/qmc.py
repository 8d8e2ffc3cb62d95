"""Python binding of the C-ABI in include/qmc.h (argument marshalling only).

Every function keeps the C name. Arrays go in as numpy arrays (host) or as
raw device pointers (ints, e.g. ``torch_tensor.data_ptr()``); streams as raw
``cudaStream_t`` values (``torch.cuda.current_stream().cuda_stream``).
All computation happens in libqmc.so; there is no Python or CPU fallback:
if the library is missing or no GPU is usable, calls raise ``QmcError``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

P = ctypes.POINTER
_lock = threading.Lock()
_lib = None

QMC_OK = 0
QMC_PRECISION_FP64 = 0
QMC_PRECISION_MIXED = 1
QMC_TRANSFORM_KOROBOV3, QMC_TRANSFORM_BAKER, QMC_TRANSFORM_NONE = 0, 1, 2
QMC_JOB_UNSHIFTED = 1
QMC_TARGET_COEFFICIENT, QMC_TARGET_AMPLITUDE = 0, 1
QMC_LATTICE_CBC, QMC_LATTICE_MEDIAN = 0, 1
QMC_DEVICE_NONE = -1
ERRORS = {-1: "QMC_E_INVAL", -2: "QMC_E_PARSE", -3: "QMC_E_CUDA", -4: "QMC_E_TIMEOUT",
          -5: "QMC_E_NOT_CONVERGED", -6: "QMC_E_SIGN_CHECK", -7: "QMC_E_NONFINITE", -8: "QMC_E_NOMEM"}


QMC_NUM_CLASSES = 13  # evaluator classes (include/qmc.h)


class QmcError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class qmc_options(ctypes.Structure):
    _fields_ = [("shifts", ctypes.c_int), ("seed", ctypes.c_uint64), ("block", ctypes.c_int),
                ("ppt", ctypes.c_int), ("min_points", ctypes.c_uint64),
                ("max_points", ctypes.c_uint64), ("presamples", ctypes.c_int),
                ("lambda_", ctypes.c_double), ("precision", ctypes.c_int),
                ("transform", ctypes.c_int), ("target_mode", ctypes.c_int),
                ("max_growth", ctypes.c_int), ("lattice", ctypes.c_int), ("lattice_candidates", ctypes.c_int),
                ("batched", ctypes.c_int), ("keep_shift_sums", ctypes.c_int), ("reserved", ctypes.c_int * 4)]


class qmc_sum_spec(ctypes.Structure):
    _fields_ = [("integral_ids", ctypes.POINTER(ctypes.c_int)), ("nint", ctypes.c_int),
                ("namp", ctypes.c_int), ("coef", ctypes.c_void_p), ("coef_lo", ctypes.c_int),
                ("ncoef", ctypes.c_int)]


class qmc_integrate_info(ctypes.Structure):
    _fields_ = [("evaluations", ctypes.c_double), ("seconds", ctypes.c_double),
                ("kernel_seconds", ctypes.c_double), ("iterations", ctypes.c_int),
                ("max_lattice", ctypes.c_uint64), ("presample_evaluations", ctypes.c_double),
                ("fp64_escalations", ctypes.c_int), ("median_evaluations", ctypes.c_double)]


class qmc_shift_layout(ctypes.Structure):
    _fields_ = [("npoints", ctypes.c_int), ("nsectors", ctypes.c_int), ("shifts", ctypes.c_int),
                ("sector_lo", ctypes.c_int), ("sector_orders", ctypes.c_int), ("count", ctypes.c_size_t)]


class qmc_job(ctypes.Structure):
    _fields_ = [("integral_id", ctypes.c_int32), ("sector", ctypes.c_int32),
                ("point", ctypes.c_int32), ("shifts", ctypes.c_int32), ("n", ctypes.c_uint64),
                ("seed", ctypes.c_uint64), ("stream", ctypes.c_uint64),
                ("lambda_", ctypes.c_double * 6), ("z", ctypes.c_uint32 * 6), ("flags", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


class qmc_c64(ctypes.Structure):
    _fields_ = [("re", ctypes.c_double), ("im", ctypes.c_double)]


# callback types of qmc_set_ranks and qmc_set_evaluator
ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_size_t)
EVAL_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(qmc_job), ctypes.c_int, ctypes.c_int,
                           ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_uint32))
_callbacks = {}   # keeps the ctypes callback objects alive per context


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libqmc.so (building it first if it is absent or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            if not os.path.exists(path):
                raise QmcError(-3, f"libqmc.so missing at {path}")
            L = ctypes.CDLL(path)
            vp, i32, u64, dbl, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_double, ctypes.c_size_t
            sig = {
                "qmc_create": ([P(vp), i32, P(qmc_options)], i32),
                "qmc_destroy": ([vp], None),
                "qmc_last_error": ([vp], ctypes.c_char_p),
                "qmc_set_lattices": ([vp, P(u64), P(ctypes.c_uint32), i32], i32),
                "qmc_load_sectors_mem": ([vp, ctypes.c_char_p, sz, P(i32)], i32),
                "qmc_load_sectors": ([vp, ctypes.c_char_p, P(i32)], i32),
                "qmc_integral_info": ([vp, i32, P(i32), P(i32), P(i32), P(qmc_c64), i32, P(i32)], i32),
                "qmc_set_kinematics": ([vp, P(dbl), i32, i32], i32),
                "qmc_plan_create": ([vp, P(qmc_job), i32, i32, i32, P(vp)], i32),
                "qmc_plan_output_size": ([vp], sz),
                "qmc_plan_run": ([vp, vp, vp], i32),
                "qmc_plan_results": ([vp, P(dbl), P(u64)], i32),
                "qmc_plan_last_time": ([vp, P(ctypes.c_float), P(ctypes.c_float), P(i32)], i32),
                "qmc_plan_destroy": ([vp], None),
                "qmc_eval_jobs": ([vp, P(qmc_job), i32, i32, i32, P(dbl)], i32),
                "qmc_lattice_points": ([vp, u64, P(ctypes.c_uint32), i32, P(dbl), u64, u64, P(dbl),
                                        P(u64)], i32),
                "qmc_shifts": ([vp, u64, u64, i32, i32, P(dbl)], i32),
                "qmc_fp64_peak": ([vp, P(dbl)], i32),
                "qmc_fp32_peak": ([vp, P(dbl)], i32),
                "qmc_eval_jobs_noalloc": ([vp, P(qmc_job), i32, i32, i32, vp, vp], i32),
                "qmc_fp64_log": ([vp, P(dbl), sz, P(dbl)], i32),
                "qmc_fp64_rcp": ([vp, P(dbl), sz, P(dbl)], i32),
                "qmc_korobov3": ([vp, P(dbl), sz, P(dbl)], i32),
                "qmc_fp64_atan2": ([vp, P(dbl), P(dbl), sz, P(dbl)], i32),
                "qmc_shift_stats": ([P(dbl), i32, i32, P(dbl), P(dbl)], i32),
                "qmc_plan_use_graph": ([vp, i32], i32),
                "qmc_plan_job_failures": ([vp, P(ctypes.c_uint32)], i32),
                "qmc_presample_lambda": ([vp, P(qmc_job), i32, i32, i32, dbl, i32], i32),
                "qmc_autotune": ([vp, P(qmc_job), i32, i32, i32, P(i32), P(i32)], i32),
                "qmc_median_candidates": ([u64, i32, i32, u64, P(ctypes.c_uint32)], i32),
                "qmc_gemm_bf16": ([P(ctypes.c_uint16), P(ctypes.c_uint16), P(ctypes.c_float), i32, i32, i32], i32),
                "qmc_gemm_bf16_device": ([vp, vp, vp, i32, i32, i32, vp, vp], i32),
                "qmc_gemm_bf16_device_limit": ([vp, vp, vp, i32, i32, i32, vp, vp, ctypes.c_uint32], i32),
                "qmc_mlp_create": ([P(vp), i32, i32, i32, i32, i32, u64], i32),
                "qmc_mlp_destroy": ([vp], None),
                "qmc_mlp_num_params": ([vp, P(sz)], i32),
                "qmc_mlp_get_params": ([vp, P(ctypes.c_float), sz], i32),
                "qmc_mlp_set_params": ([vp, P(ctypes.c_float), sz], i32),
                "qmc_mlp_forward": ([vp, P(ctypes.c_float), i32, P(ctypes.c_float)], i32),
                "qmc_mlp_grad": ([vp, P(ctypes.c_float), P(ctypes.c_float), P(ctypes.c_float), i32,
                                  P(ctypes.c_float), P(ctypes.c_float)], i32),
                "qmc_mlp_train": ([vp, P(ctypes.c_float), P(ctypes.c_float), P(ctypes.c_float), i32, i32,
                                   ctypes.c_float, P(ctypes.c_float)], i32),
                "qmc_median_lattice": ([vp, P(qmc_job), i32, i32, i32, u64, P(ctypes.c_uint32), P(dbl)], i32),
                "qmc_series_mul": ([P(qmc_c64), i32, i32, P(qmc_c64), i32, i32, i32, i32, P(qmc_c64)], i32),
                "qmc_series_var": ([P(qmc_c64), i32, i32, P(dbl), i32, i32, i32, i32, P(dbl)], i32),
                "qmc_allocate": ([P(dbl), P(dbl), P(dbl), i32, i32, dbl, dbl, P(dbl)], i32),
                "qmc_integrate": ([vp, P(qmc_sum_spec), dbl, dbl, dbl, i32, i32, P(qmc_c64), P(qmc_c64),
                                   P(qmc_integrate_info)], i32),
                "qmc_integrate_ex": ([vp, P(qmc_sum_spec), dbl, dbl, dbl, i32, i32, P(qmc_c64), P(qmc_c64),
                                      P(qmc_integrate_info), P(u64), i32, P(dbl), P(u64), P(dbl)], i32),
                "qmc_set_coefficients": ([vp, i32, P(qmc_c64), i32, i32, i32, i32], i32),
                "qmc_integral_results": ([vp, i32, P(qmc_c64), P(qmc_c64)], i32),
                "qmc_per_shift_sums": ([vp, i32, P(dbl), sz, P(qmc_shift_layout), P(u64)], i32),
                "qmc_stats": ([vp, P(dbl), P(dbl)], i32),
                "qmc_set_ranks": ([vp, i32, i32, ALLREDUCE_FN, vp], i32),
                "qmc_set_evaluator": ([vp, EVAL_FN, vp], i32),
            }
            for name, (args, res) in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def exported_symbols():
    """Names of the C-ABI functions this binding expects libqmc.so to export."""
    return ["qmc_create", "qmc_destroy", "qmc_last_error", "qmc_set_lattices",
            "qmc_load_sectors_mem", "qmc_load_sectors", "qmc_integral_info", "qmc_set_kinematics",
            "qmc_plan_create", "qmc_plan_output_size", "qmc_plan_run", "qmc_plan_results",
            "qmc_plan_last_time", "qmc_plan_destroy", "qmc_eval_jobs", "qmc_lattice_points",
            "qmc_shifts", "qmc_fp64_peak", "qmc_fp32_peak", "qmc_eval_jobs_noalloc", "qmc_fp64_log", "qmc_fp64_rcp", "qmc_korobov3", "qmc_fp64_atan2",
            "qmc_shift_stats", "qmc_series_mul", "qmc_series_var", "qmc_allocate", "qmc_integrate",
            "qmc_plan_use_graph", "qmc_plan_job_failures", "qmc_presample_lambda", "qmc_autotune",
            "qmc_median_candidates", "qmc_median_lattice", "qmc_gemm_bf16", "qmc_gemm_bf16_device",
            "qmc_gemm_bf16_device_limit", "qmc_mlp_create",
            "qmc_mlp_destroy", "qmc_mlp_num_params", "qmc_mlp_get_params", "qmc_mlp_set_params",
            "qmc_mlp_forward", "qmc_mlp_grad", "qmc_mlp_train", "qmc_integrate_ex", "qmc_set_coefficients",
            "qmc_integral_results", "qmc_per_shift_sums", "qmc_stats", "qmc_set_ranks", "qmc_set_evaluator"]


def _dp(a):
    return a.ctypes.data_as(P(ctypes.c_double))


def _check(ctx, rc):
    if rc != QMC_OK:
        msg = lib().qmc_last_error(ctx).decode() if ctx else ""
        raise QmcError(rc, msg)


# ------------------------------------------------------------------ C names
def qmc_create(device: int = 0, **opts):
    o = qmc_options()
    for k, v in opts.items():
        setattr(o, "lambda_" if k == "lambda" else k, v)
    h = ctypes.c_void_p()
    rc = lib().qmc_create(ctypes.byref(h), device, ctypes.byref(o))
    if rc != QMC_OK:
        raise QmcError(rc, "qmc_create failed (no usable CUDA device?)" if rc == -3 else "qmc_create failed")
    return h


def qmc_destroy(ctx):
    lib().qmc_destroy(ctx)
    _callbacks.pop(ctx.value if isinstance(ctx, ctypes.c_void_p) else ctx, None)


def qmc_last_error(ctx) -> str:
    return lib().qmc_last_error(ctx).decode()


def qmc_set_lattices(ctx, n, z):
    n = np.ascontiguousarray(n, dtype=np.uint64)
    z = np.ascontiguousarray(z, dtype=np.uint32).reshape(len(n), 6)
    _check(ctx, lib().qmc_set_lattices(ctx, n.ctypes.data_as(P(ctypes.c_uint64)),
                                       z.ctypes.data_as(P(ctypes.c_uint32)), len(n)))


def qmc_load_sectors_mem(ctx, text: str) -> int:
    b = text.encode()
    iid = ctypes.c_int()
    _check(ctx, lib().qmc_load_sectors_mem(ctx, b, len(b), ctypes.byref(iid)))
    return iid.value


def qmc_load_sectors(ctx, path: str) -> int:
    iid = ctypes.c_int()
    _check(ctx, lib().qmc_load_sectors(ctx, path.encode(), ctypes.byref(iid)))
    return iid.value


def qmc_integral_info(ctx, integral_id: int):
    ns, mp, lo, ln = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    buf = (qmc_c64 * 64)()
    _check(ctx, lib().qmc_integral_info(ctx, integral_id, ctypes.byref(ns), ctypes.byref(mp),
                                        ctypes.byref(lo), buf, 64, ctypes.byref(ln)))
    return ns.value, mp.value, lo.value, [complex(buf[i].re, buf[i].im) for i in range(ln.value)]


def qmc_set_kinematics(ctx, inv):
    inv = np.ascontiguousarray(inv, dtype=np.float64)
    if inv.ndim == 1:
        inv = inv.reshape(-1, 1) if inv.size else inv.reshape(0, 0)
    npts, ninv = inv.shape
    _check(ctx, lib().qmc_set_kinematics(ctx, _dp(inv), npts, ninv))


def make_jobs(specs):
    """specs: iterable of dicts with integral_id, sector, point, shifts, n, seed, stream, lambda."""
    specs = list(specs)
    arr = (qmc_job * max(1, len(specs)))()
    for i, s in enumerate(specs):
        arr[i].integral_id = s["integral_id"]
        arr[i].sector = s["sector"]
        arr[i].point = s.get("point", 0)
        arr[i].shifts = s["shifts"]
        arr[i].n = s["n"]
        arr[i].seed = s.get("seed", 1)
        arr[i].stream = s.get("stream", 0)
        lam = np.broadcast_to(np.asarray(s.get("lambda", 0.0), dtype=np.float64), (6,))
        for j in range(6):
            arr[i].lambda_[j] = float(lam[j])
        z = s.get("z")
        if z is not None:
            for j in range(6):
                arr[i].z[j] = int(z[j]) if j < len(z) else 1
        arr[i].flags = int(s.get("flags", 0))
    return arr, len(specs)


def qmc_plan_create(ctx, jobs, njobs: int, lo: int, norders: int):
    h = ctypes.c_void_p()
    _check(ctx, lib().qmc_plan_create(ctx, jobs, njobs, lo, norders, ctypes.byref(h)))
    return h


def qmc_plan_output_size(plan) -> int:
    return lib().qmc_plan_output_size(plan)


def qmc_plan_run(ctx, plan, out_dev_ptr=None, stream_ptr=None):
    _check(ctx, lib().qmc_plan_run(plan, ctypes.c_void_p(out_dev_ptr or 0) if out_dev_ptr else None,
                                   ctypes.c_void_p(stream_ptr) if stream_ptr else None))


def qmc_plan_results(ctx, plan, out=None, check=True):
    size = qmc_plan_output_size(plan)
    if out is None:
        out = np.zeros(size, dtype=np.float64)
    fails = ctypes.c_uint64()
    rc = lib().qmc_plan_results(plan, _dp(out) if size else None, ctypes.byref(fails))
    if check:
        _check(ctx, rc)
    return out, fails.value, rc


def qmc_plan_last_time(ctx, plan):
    ms, mse, nl = ctypes.c_float(), ctypes.c_float(), ctypes.c_int()
    _check(ctx, lib().qmc_plan_last_time(plan, ctypes.byref(ms), ctypes.byref(mse), ctypes.byref(nl)))
    return ms.value, mse.value, nl.value


def qmc_plan_use_graph(ctx, plan, enable=True):
    _check(ctx, lib().qmc_plan_use_graph(plan, 1 if enable else 0))


def qmc_plan_job_failures(ctx, plan, njobs):
    out = np.zeros(njobs, dtype=np.uint32)
    _check(ctx, lib().qmc_plan_job_failures(plan, out.ctypes.data_as(P(ctypes.c_uint32))))
    return out


def qmc_presample_lambda(ctx, jobs, njobs, lo, norders, lambda_max=1.0, ncand=12, check=True):
    """Choose lambda per deformed job in place (jobs is the ctypes array from make_jobs)."""
    rc = lib().qmc_presample_lambda(ctx, jobs, njobs, lo, norders, lambda_max, ncand)
    if check:
        _check(ctx, rc)
    return np.array([jobs[i].lambda_[0] for i in range(njobs)]), rc


def qmc_autotune(ctx, jobs, njobs, lo, norders):
    bb = (ctypes.c_int * QMC_NUM_CLASSES)()
    bp = (ctypes.c_int * QMC_NUM_CLASSES)()
    _check(ctx, lib().qmc_autotune(ctx, jobs, njobs, lo, norders, bb, bp))
    return list(bb), list(bp)


def qmc_median_candidates(n, d, r, seed):
    z = np.zeros((r, 6), dtype=np.uint32)
    _check(None, lib().qmc_median_candidates(n, d, r, seed, z.ctypes.data_as(P(ctypes.c_uint32))))
    return z


def qmc_median_lattice(ctx, job_spec, lo, norders, r, seed):
    """(z [6], per-candidate estimates [r][norders][2]) for one job spec dict."""
    jobs, _ = make_jobs([job_spec])
    z = np.zeros(6, dtype=np.uint32)
    est = np.zeros((r, norders, 2))
    _check(ctx, lib().qmc_median_lattice(ctx, jobs, lo, norders, r, seed, z.ctypes.data_as(P(ctypes.c_uint32)),
                                         _dp(est)))
    return z, est


def to_bf16_bits(x):
    """Round float32 values to bfloat16 (nearest even) and return the 16-bit patterns."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)
    return r


def from_bf16_bits(b):
    return (np.ascontiguousarray(b, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32)


def qmc_gemm_bf16(A_bits, B_bits):
    """C = A B^T on the tensor cores; A [M][K], B [N][K] bf16 bit patterns."""
    A_bits = np.ascontiguousarray(A_bits, dtype=np.uint16)
    B_bits = np.ascontiguousarray(B_bits, dtype=np.uint16)
    M, K = A_bits.shape
    N = B_bits.shape[0]
    C = np.zeros((M, N), dtype=np.float32)
    _check(None, lib().qmc_gemm_bf16(A_bits.ctypes.data_as(P(ctypes.c_uint16)),
                                     B_bits.ctypes.data_as(P(ctypes.c_uint16)),
                                     C.ctypes.data_as(P(ctypes.c_float)), M, N, K))
    return C


def qmc_gemm_bf16_device(A_ptr, B_ptr, C_ptr, M, N, K, err_ptr, stream_ptr=0):
    """The same GEMM on device pointers (e.g. torch data_ptr()), enqueued on
    `stream_ptr`; err_ptr points at a caller-zeroed device unsigned."""
    _check(None, lib().qmc_gemm_bf16_device(ctypes.c_void_p(A_ptr), ctypes.c_void_p(B_ptr), ctypes.c_void_p(C_ptr),
                                            M, N, K, ctypes.c_void_p(err_ptr),
                                            ctypes.c_void_p(stream_ptr) if stream_ptr else None))


def qmc_gemm_bf16_device_limit(A_ptr, B_ptr, C_ptr, M, N, K, err_ptr, wait_limit, stream_ptr=0):
    """qmc_gemm_bf16_device with `wait_limit` polls per pipeline wait."""
    _check(None, lib().qmc_gemm_bf16_device_limit(ctypes.c_void_p(A_ptr), ctypes.c_void_p(B_ptr),
                                                  ctypes.c_void_p(C_ptr), M, N, K, ctypes.c_void_p(err_ptr),
                                                  ctypes.c_void_p(stream_ptr) if stream_ptr else None,
                                                  int(wait_limit)))


def _fp(a):
    return a.ctypes.data_as(P(ctypes.c_float))


class Mlp:
    """The C-ABI's tensor-core MLP (qmc_mlp_*), host numpy in and out."""

    def __init__(self, nin, width, depth, nout, seed=1, device=0):
        self.h = ctypes.c_void_p()
        rc = lib().qmc_mlp_create(ctypes.byref(self.h), device, nin, width, depth, nout, seed)
        if rc:
            raise QmcError(rc, "qmc_mlp_create failed")
        self.shape = (nin, width, depth, nout)
        n = ctypes.c_size_t()
        lib().qmc_mlp_num_params(self.h, ctypes.byref(n))
        self.nparams = n.value

    def close(self):
        if self.h:
            lib().qmc_mlp_destroy(self.h)
            self.h = None

    def params(self):
        p = np.zeros(self.nparams, dtype=np.float32)
        _check(None, lib().qmc_mlp_get_params(self.h, _fp(p), self.nparams))
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(None, lib().qmc_mlp_set_params(self.h, _fp(p), self.nparams))

    def forward(self, x):
        x = np.ascontiguousarray(x, dtype=np.float32)
        y = np.zeros((x.shape[0], self.shape[3]), dtype=np.float32)
        _check(None, lib().qmc_mlp_forward(self.h, _fp(x), x.shape[0], _fp(y)))
        return y

    def grad(self, x, y, wt=None):
        x = np.ascontiguousarray(x, dtype=np.float32)
        y = np.ascontiguousarray(y, dtype=np.float32)
        w = None if wt is None else np.ascontiguousarray(wt, dtype=np.float32)
        loss = ctypes.c_float()
        g = np.zeros(self.nparams, dtype=np.float32)
        _check(None, lib().qmc_mlp_grad(self.h, _fp(x), _fp(y), _fp(w) if w is not None else None, x.shape[0],
                                        ctypes.byref(loss), _fp(g)))
        return loss.value, g

    def train(self, x, y, steps, lr, wt=None):
        x = np.ascontiguousarray(x, dtype=np.float32)
        y = np.ascontiguousarray(y, dtype=np.float32)
        w = None if wt is None else np.ascontiguousarray(wt, dtype=np.float32)
        losses = np.zeros(max(1, steps), dtype=np.float32)
        _check(None, lib().qmc_mlp_train(self.h, _fp(x), _fp(y), _fp(w) if w is not None else None, x.shape[0],
                                         steps, lr, _fp(losses)))
        return losses[:steps]


def qmc_plan_destroy(plan):
    lib().qmc_plan_destroy(plan)


def qmc_eval_jobs(ctx, jobs, njobs: int, lo: int, norders: int, size: int):
    out = np.zeros(size, dtype=np.float64)
    _check(ctx, lib().qmc_eval_jobs(ctx, jobs, njobs, lo, norders, _dp(out)))
    return out


def qmc_lattice_points(ctx, n: int, z, delta, k0: int, count: int):
    z = np.ascontiguousarray(z, dtype=np.uint32)
    d = len(z)
    delta = np.ascontiguousarray(delta, dtype=np.float64).reshape(d)
    x = np.zeros((count, d), dtype=np.float64)
    r = np.zeros((count, d), dtype=np.uint64)
    _check(ctx, lib().qmc_lattice_points(ctx, n, z.ctypes.data_as(P(ctypes.c_uint32)), d, _dp(delta),
                                         k0, count, _dp(x), r.ctypes.data_as(P(ctypes.c_uint64))))
    return x, r


def qmc_shifts(ctx, seed: int, stream: int, m: int, d: int):
    out = np.zeros((m, d), dtype=np.float64)
    _check(ctx, lib().qmc_shifts(ctx, seed, stream, m, d, _dp(out)))
    return out


def qmc_eval_jobs_noalloc(ctx, jobs, njobs: int, lo: int, norders: int, out_dev_ptr: int,
                          stream_ptr=None):
    """Evaluate into a caller-owned device buffer without allocating (see qmc.h)."""
    _check(ctx, lib().qmc_eval_jobs_noalloc(ctx, jobs, njobs, lo, norders, ctypes.c_void_p(out_dev_ptr),
                                            ctypes.c_void_p(stream_ptr) if stream_ptr else None))


def qmc_fp64_log(ctx, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    _check(ctx, lib().qmc_fp64_log(ctx, _dp(x), x.size, _dp(out)))
    return out


def qmc_fp64_atan2(ctx, y, x):
    y = np.ascontiguousarray(y, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    _check(ctx, lib().qmc_fp64_atan2(ctx, _dp(y), _dp(x), x.size, _dp(out)))
    return out


def qmc_korobov3(ctx, u):
    """(t, 1 - t, u (1 - u)) of the evaluator's korobov3 transform at each u."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros((u.size, 3))
    _check(ctx, lib().qmc_korobov3(ctx, _dp(u), u.size, _dp(out)))
    return out[:, 0].copy(), out[:, 1].copy(), out[:, 2].copy()


def qmc_fp64_rcp(ctx, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    _check(ctx, lib().qmc_fp64_rcp(ctx, _dp(x), x.size, _dp(out)))
    return out


def _c64(a):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a, a.ctypes.data_as(P(qmc_c64))


def qmc_shift_stats(sums):
    """sums [m][norders][2] -> (mean [norders][2], variance of the mean [norders][2])."""
    sums = np.ascontiguousarray(sums, dtype=np.float64)
    m, no = sums.shape[0], sums.shape[1]
    mean = np.zeros((no, 2))
    var = np.zeros((no, 2))
    _check(None, lib().qmc_shift_stats(_dp(sums), m, no, _dp(mean), _dp(var)))
    return mean, var


def qmc_series_mul(a, a_lo, b, b_lo, lo, n):
    a, pa = _c64(a)
    b, pb = _c64(b)
    out = np.zeros(n, dtype=np.complex128)
    _check(None, lib().qmc_series_mul(pa, a_lo, len(a), pb, b_lo, len(b), lo, n,
                                      out.ctypes.data_as(P(qmc_c64))))
    return out


def qmc_series_var(c, c_lo, v, v_lo, lo, n):
    c, pc = _c64(c)
    v = np.ascontiguousarray(v, dtype=np.float64)
    out = np.zeros(n)
    _check(None, lib().qmc_series_var(pc, c_lo, len(c), _dp(v), v_lo, len(v), lo, n, _dp(out)))
    return out


def qmc_allocate(W, tau, V, alpha=2.0, n_min=0.0):
    """W [nsums][nint], tau [nint], V [nsums] -> n [nint] (Eq. adaptive-solution)."""
    W = np.ascontiguousarray(np.atleast_2d(W), dtype=np.float64)
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    V = np.ascontiguousarray(np.atleast_1d(V), dtype=np.float64)
    out = np.zeros(W.shape[1])
    _check(None, lib().qmc_allocate(_dp(W), _dp(tau), _dp(V), W.shape[0], W.shape[1], alpha, n_min,
                                    _dp(out)))
    return out


def qmc_integrate(ctx, integral_ids=None, coef=None, coef_lo=0, epsrel=1e-4, epsabs=0.0, timeout=0.0,
                  lowest_order=0, norders=1, npoints=1, namp=1, check=True, n_init=None, shifts=0,
                  nslots=0, lambda_io=None):
    """Adaptive integration; returns (value, error, info dict, return code), and with
    ``nslots`` > 0 also (w_out, n_out) per (point, integral, sector) slot.
    value/error: complex [npoints][namp][norders] (error = sigma_re + 1j sigma_im)."""
    spec = None
    keep = []
    if integral_ids is not None:
        ids = (ctypes.c_int * len(integral_ids))(*integral_ids)
        keep.append(ids)
        spec = qmc_sum_spec()
        spec.integral_ids = ids
        spec.nint = len(integral_ids)
        spec.namp = namp
        if coef is not None:
            c = np.ascontiguousarray(coef, dtype=np.complex128)
            keep.append(c)
            spec.coef = c.ctypes.data
            spec.coef_lo = coef_lo
            spec.ncoef = c.shape[-1]
    value = np.zeros((npoints, namp, norders), dtype=np.complex128)
    error = np.zeros((npoints, namp, norders), dtype=np.complex128)
    info = qmc_integrate_info()
    w_out = np.zeros(max(1, nslots))
    n_out = np.zeros(max(1, nslots), dtype=np.uint64)
    ni = None
    if n_init is not None:
        ni = np.ascontiguousarray(n_init, dtype=np.uint64)
        keep.append(ni)
    rc = lib().qmc_integrate_ex(ctx, ctypes.byref(spec) if spec is not None else None, epsrel, epsabs, timeout,
                                lowest_order, norders, value.ctypes.data_as(P(qmc_c64)),
                                error.ctypes.data_as(P(qmc_c64)), ctypes.byref(info),
                                ni.ctypes.data_as(P(ctypes.c_uint64)) if ni is not None else None, shifts,
                                _dp(w_out) if nslots else None,
                                n_out.ctypes.data_as(P(ctypes.c_uint64)) if nslots else None,
                                _dp(lambda_io) if lambda_io is not None else None)
    if check and rc not in (0,):
        _check(ctx, rc)
    d = {k: getattr(info, k) for k, _ in qmc_integrate_info._fields_}
    if nslots:
        return value, error, d, rc, w_out[:nslots], n_out[:nslots]
    return value, error, d, rc


def qmc_set_coefficients(ctx, coef, coef_lo=0):
    """coef: complex [npoints][namp][nint][ncoef] over all loaded integrals
    (None clears them)."""
    if coef is None:
        _check(ctx, lib().qmc_set_coefficients(ctx, 0, None, 0, 0, 0, 0))
        return
    c, pc = _c64(coef)
    npts, namp, nint, nc = c.shape
    _check(ctx, lib().qmc_set_coefficients(ctx, namp, pc, npts, nint, coef_lo, nc))


def qmc_integral_results(ctx, integral_id, npoints, norders):
    """(value, error) complex [npoints][norders] of one integral from the last qmc_integrate."""
    v = np.zeros((npoints, norders), dtype=np.complex128)
    e = np.zeros((npoints, norders), dtype=np.complex128)
    _check(ctx, lib().qmc_integral_results(ctx, integral_id, v.ctypes.data_as(P(qmc_c64)),
                                           e.ctypes.data_as(P(qmc_c64))))
    return v, e


def qmc_per_shift_sums(ctx, integral_id):
    """(sums [npoints][nsectors][shifts][sector_orders][2], sector_lo, n [npoints][nsectors])."""
    lay = qmc_shift_layout()
    _check(ctx, lib().qmc_per_shift_sums(ctx, integral_id, None, 0, ctypes.byref(lay), None))
    out = np.zeros(lay.count)
    n = np.zeros(lay.npoints * lay.nsectors, dtype=np.uint64)
    _check(ctx, lib().qmc_per_shift_sums(ctx, integral_id, _dp(out), out.size, None,
                                         n.ctypes.data_as(P(ctypes.c_uint64))))
    return (out.reshape(lay.npoints, lay.nsectors, lay.shifts, lay.sector_orders, 2), lay.sector_lo,
            n.reshape(lay.npoints, lay.nsectors))


def qmc_stats(ctx):
    e, sec = ctypes.c_double(), ctypes.c_double()
    _check(ctx, lib().qmc_stats(ctx, ctypes.byref(e), ctypes.byref(sec)))
    return e.value, sec.value


def _key(ctx):
    return ctx.value if isinstance(ctx, ctypes.c_void_p) else ctx


def qmc_set_ranks(ctx, rank, world, allreduce):
    """allreduce(buf: numpy float64 array view) sums buf over the ranks in place."""
    if allreduce is None or world == 1:
        _check(ctx, lib().qmc_set_ranks(ctx, 0, 1, ALLREDUCE_FN(), None))
        _callbacks.get(_key(ctx), {}).pop("allreduce", None)
        return

    def cb(user, buf, n):
        try:
            arr = np.ctypeslib.as_array(buf, shape=(n,))
            allreduce(arr)
            return 0
        except Exception:   # noqa: BLE001 -- reported to the library as a failed exchange
            return -1

    f = ALLREDUCE_FN(cb)
    _callbacks.setdefault(_key(ctx), {})["allreduce"] = f
    _check(ctx, lib().qmc_set_ranks(ctx, rank, world, f, None))


def qmc_set_evaluator(ctx, evaluate):
    """evaluate(jobs: list of dicts, lo, norders) -> (out [njobs][shifts][norders][2], fails [njobs] or None)
    replaces the GPU evaluator of qmc_integrate (None restores it)."""
    if evaluate is None:
        _check(ctx, lib().qmc_set_evaluator(ctx, EVAL_FN(), None))
        _callbacks.get(_key(ctx), {}).pop("eval", None)
        return

    def cb(user, jobs, njobs, lo, norders, out, fails):
        try:
            specs = []
            for i in range(njobs):
                J = jobs[i]
                specs.append(dict(integral_id=J.integral_id, sector=J.sector, point=J.point, shifts=J.shifts,
                                  n=J.n, seed=J.seed, stream=J.stream, flags=J.flags,
                                  z=[J.z[j] for j in range(6)], **{"lambda": [J.lambda_[j] for j in range(6)]}))
            vals, fl = evaluate(specs, lo, norders)
            flat = np.concatenate([np.asarray(v, dtype=np.float64).ravel() for v in vals]) if vals else np.zeros(0)
            dst = np.ctypeslib.as_array(out, shape=(flat.size,)) if flat.size else None
            if dst is not None:
                dst[:] = flat
            if fl is not None and any(fl):
                fdst = np.ctypeslib.as_array(fails, shape=(njobs,))
                fdst[:] = np.asarray(fl, dtype=np.uint32)
                return -6
            return 0
        except Exception:   # noqa: BLE001 -- reported to the library as a failed evaluation
            import traceback

            traceback.print_exc()
            return -1

    f = EVAL_FN(cb)
    _callbacks.setdefault(_key(ctx), {})["eval"] = f
    _check(ctx, lib().qmc_set_evaluator(ctx, f, None))


def qmc_fp64_peak(ctx) -> float:
    g = ctypes.c_double()
    _check(ctx, lib().qmc_fp64_peak(ctx, ctypes.byref(g)))
    return g.value


def qmc_fp32_peak(ctx) -> float:
    g = ctypes.c_double()
    _check(ctx, lib().qmc_fp32_peak(ctx, ctypes.byref(g)))
    return g.value


# ------------------------------------------------------------------ helpers
def load_lattice_table(ctx):
    """Install the committed CBC table (inputs/cbc_table.txt) into a context."""
    from .inputs.lattice import load_table

    rows = load_table()
    n = np.array([r[0] for r in rows], dtype=np.uint64)
    z = np.array([list(r[1]) + [1] * (6 - len(r[1])) for r in rows], dtype=np.uint32)
    qmc_set_lattices(ctx, n, z)
    return rows


def jobs_for_integral(integral_id: int, nsectors: int, npoints: int, n: int, shifts: int, seed=1,
                      lam=0.0, stream_base: int = 0):
    """One job per (point, sector); shift stream id = stream_base + point * nsectors + sector."""
    specs = []
    for p in range(npoints):
        for s in range(nsectors):
            L = lam[p][s] if hasattr(lam, "__len__") else lam
            specs.append(dict(integral_id=integral_id, sector=s, point=p, shifts=shifts, n=n,
                              seed=seed, stream=stream_base + p * nsectors + s, **{"lambda": L}))
    return specs
