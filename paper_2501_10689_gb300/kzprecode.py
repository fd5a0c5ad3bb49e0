"""ctypes binding of libkzprecode (argument marshalling only).

Every function named like a C entry point takes the same arguments, with
torch CUDA tensors in place of device pointers and NumPy int32 arrays in place
of host arrays, and returns what the C call returns (raising ``KzError`` on a
non-OK status).  All arithmetic runs in the CUDA library; when the shared
library is missing this module raises instead of falling back to anything.

Layouts: a K x nrhs column-major matrix is a contiguous torch tensor of shape
(nrhs, K) (one row per right-hand side); likewise x is (nrhs, Nt).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import _build

# enums of include/kzprecode.h
KZ_OK, KZ_NOT_CONVERGED, KZ_ERR_INVALID_ARG, KZ_ERR_NUMERIC, KZ_ERR_CUDA, KZ_ERR_NOMEM, KZ_ERR_UNSUPPORTED = range(7)
KZ_STATUS_BIT_NOT_CONVERGED, KZ_STATUS_BIT_NUMERIC, KZ_STATUS_BIT_TIMEOUT = 1, 2, 4
ALGOS = {"rk_energy": 0, "rk_uniform": 1, "grk": 2, "ahk": 3, "vr_ogrk": 4, "vr_oahk": 5, "rk_swor": 6, "gk": 7}
SELECT = {"paper": 0, "baiwu": 1, "argmax": 2}
PREC = {"c64": 0, "bf16": 1}

_lib = None


class KzError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libkzprecode status {code}: {msg}")
        self.code = code


class KzAdjointItem(ctypes.Structure):
    _fields_ = [("Q", ctypes.c_void_p), ("X", ctypes.c_void_p), ("G_Q", ctypes.c_void_p), ("G_X", ctypes.c_void_p),
                ("grad_H_packed", ctypes.c_void_p), ("grad_xi", ctypes.c_void_p)]


class KzBatchItem(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("s", ctypes.c_void_p), ("x", ctypes.c_void_p),
                ("v", ctypes.c_void_p), ("iters", ctypes.c_void_p), ("resid", ctypes.c_void_p),
                ("xi", ctypes.c_float)]


EXPORTS = ("kz_plan_create", "kz_plan_dense", "kz_plan_update", "kz_plan_destroy", "kz_plan_query", "kz_precode", "kz_precode_ex",
           "kz_batch_prepare", "kz_precode_batched", "kz_batch_destroy", "kz_batch_tune", "kz_batch_set_launch",
           "kz_batch_query",
           "kz_batch_rebind", "kz_batch_update", "kz_batch_update_items", "kz_precode_adjoint", "kz_precode_adjoint_batched", "kz_precode_adjoint_noalloc",
           "kz_precode_record", "kz_unrolled_adjoint", "kz_precoder_matrix", "kz_plan_flops", "kz_sum_rate", "kz_sum_rate_batched", "kz_last_error", "kz_version")
KERNELS = {"auto": 0, "resident": 1, "tc": 3, "group": 4, "small": 5}


def library_path() -> str:
    return _build.lib_path()


def load():
    """Load the shared library (built by ``_build.build``); raise if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P, I32, I64, F32, F64, U64 = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float,
                                  ctypes.c_double, ctypes.c_uint64)
    lib.kz_plan_create.argtypes = [ctypes.POINTER(P), I32, I32, P, P, P, I32, P]
    lib.kz_plan_create.restype = I32
    lib.kz_plan_dense.argtypes = [ctypes.POINTER(P), I32, I32, P, P, P, I32, P]
    lib.kz_plan_dense.restype = I32
    lib.kz_precode_record.argtypes = [P, P, I32, F32, I32, I32, I32, U64, P, P, P, P, P, P, P, P]
    lib.kz_precode_record.restype = I32
    lib.kz_unrolled_adjoint.argtypes = [P, I32, F32, I32, P, P, P, P, P, P, P, P, P, P, P]
    lib.kz_unrolled_adjoint.restype = I32
    lib.kz_plan_flops.argtypes = [P, I32, I32, F64, P]
    lib.kz_plan_flops.restype = I32
    lib.kz_precoder_matrix.argtypes = [P, P, I32, I32, I32, P, P, P]
    lib.kz_precoder_matrix.restype = I32
    lib.kz_sum_rate.argtypes = [P, P, F64, P, P, P]
    lib.kz_sum_rate.restype = I32
    lib.kz_sum_rate_batched.argtypes = [P, F64, P, P, P]
    lib.kz_sum_rate_batched.restype = I32
    lib.kz_batch_rebind.argtypes = [P, P, P]
    lib.kz_batch_rebind.restype = I32
    lib.kz_batch_update.argtypes = [P, P, P]
    lib.kz_batch_update.restype = I32
    lib.kz_batch_update_items.argtypes = [P, P, I32, I32, P]
    lib.kz_batch_update_items.restype = I32
    lib.kz_plan_update.argtypes = [P, P, P]
    lib.kz_plan_update.restype = I32
    lib.kz_precode_adjoint_batched.argtypes = [P, P, F64, I32, P, P]
    lib.kz_precode_adjoint_batched.restype = I32
    lib.kz_plan_destroy.argtypes = [P]
    lib.kz_plan_destroy.restype = None
    lib.kz_plan_query.argtypes = [P, P, P, P, P, P, P, P]
    lib.kz_plan_query.restype = I32
    lib.kz_precode.argtypes = [P, P, I32, F32, I32, I32, F64, I32, U64, P, P, P, P, P, I32, I32, P]
    lib.kz_precode.restype = I32
    lib.kz_precode_ex.argtypes = [P, P, I32, F32, I32, I32, F64, I32, U64, P, P, P, P, P, I32, I32, I32, P]
    lib.kz_precode_ex.restype = I32
    lib.kz_batch_set_launch.argtypes = [P, I32, I32, I32, P]
    lib.kz_batch_set_launch.restype = I32
    lib.kz_batch_query.argtypes = [P, P, P, P, P]
    lib.kz_batch_query.restype = I32
    lib.kz_batch_prepare.argtypes = [ctypes.POINTER(P), P, I32, I32, I32, I32, I32, P]
    lib.kz_batch_prepare.restype = I32
    lib.kz_precode_batched.argtypes = [P, I32, F64, I32, U64, I32, P, P]
    lib.kz_precode_batched.restype = I32
    lib.kz_batch_destroy.argtypes = [P]
    lib.kz_batch_destroy.restype = None
    lib.kz_batch_tune.argtypes = [P, I32, F64, I32, U64, P, P]
    lib.kz_batch_tune.restype = I32
    lib.kz_precode_adjoint.argtypes = [P, I32, F32, P, P, P, P, F64, I32, P, P, P, P, P, P, P, P]
    lib.kz_precode_adjoint.restype = I32
    lib.kz_precode_adjoint_noalloc.argtypes = [P, I32, F32, P, P, P, P, F64, I32, P, P, P, P, P, P, P, P]
    lib.kz_precode_adjoint_noalloc.restype = I32
    lib.kz_last_error.argtypes = []
    lib.kz_last_error.restype = ctypes.c_char_p
    lib.kz_version.argtypes = []
    lib.kz_version.restype = I32
    _lib = lib
    return lib


def _check(code):
    if code not in (KZ_OK,):
        raise KzError(code, load().kz_last_error().decode())
    return code


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        if not t.is_cuda:
            raise ValueError("expected a CUDA tensor")
        if not t.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        return ctypes.c_void_p(t.data_ptr())
    return t


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _check_c64(t, shape, name):
    if t.dtype != torch.complex64 or tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: expected complex64 tensor of shape {tuple(shape)}, got {t.dtype} {tuple(t.shape)}")


class Plan:
    """Owner of a ``kz_plan*``."""

    def __init__(self, handle, K, Nt, sum_len, prec):
        self.handle = handle
        self.K, self.Nt, self.sum_len, self.prec = K, Nt, sum_len, prec

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.kz_plan_destroy(self.handle)
            self.handle = None


def kz_plan_create(K, Nt, vr_offset, vr_len, H_packed, prec="c64", stream=None) -> Plan:
    lib = load()
    off = np.ascontiguousarray(vr_offset, dtype=np.int32)
    ln = np.ascontiguousarray(vr_len, dtype=np.int32)
    if off.shape != (K,) or ln.shape != (K,):
        raise ValueError("vr_offset and vr_len must have K entries")
    _check_c64(H_packed, (int(ln.sum()),), "H_packed")
    h = ctypes.c_void_p()
    _check(lib.kz_plan_create(ctypes.byref(h), K, Nt, off.ctypes.data_as(ctypes.c_void_p),
                              ln.ctypes.data_as(ctypes.c_void_p), _ptr(H_packed), PREC[prec], _stream(stream)))
    return Plan(h, K, Nt, int(ln.sum()), prec)


def kz_plan_dense(K, Nt, vr_offset, vr_len, H_dense, prec="c64", stream=None) -> Plan:
    """Plan from a dense (K, Nt) complex64 CUDA tensor (only VR entries are read)."""
    lib = load()
    off = np.ascontiguousarray(vr_offset, dtype=np.int32)
    ln = np.ascontiguousarray(vr_len, dtype=np.int32)
    if off.shape != (K,) or ln.shape != (K,):
        raise ValueError("vr_offset and vr_len must have K entries")
    _check_c64(H_dense, (K, Nt), "H_dense")
    h = ctypes.c_void_p()
    _check(lib.kz_plan_dense(ctypes.byref(h), K, Nt, off.ctypes.data_as(ctypes.c_void_p),
                             ln.ctypes.data_as(ctypes.c_void_p), _ptr(H_dense), PREC[prec], _stream(stream)))
    return Plan(h, K, Nt, int(ln.sum()), prec)


def kz_plan_update(plan: Plan, H_packed, stream=None):
    lib = load()
    _check_c64(H_packed, (plan.sum_len,), "H_packed")
    return _check(lib.kz_plan_update(plan.handle, _ptr(H_packed), _stream(stream)))


def kz_plan_query(plan: Plan):
    lib = load()
    K = plan.K
    nF = ctypes.c_int32()
    F = np.zeros(K, dtype=np.int32)
    xptr = np.zeros(K + 1, dtype=np.int32)
    xidx = np.zeros(K * K, dtype=np.int32)
    _check(lib.kz_plan_query(plan.handle, None, None, None, ctypes.byref(nF), F.ctypes.data_as(ctypes.c_void_p),
                             xptr.ctypes.data_as(ctypes.c_void_p), xidx.ctypes.data_as(ctypes.c_void_p)))
    return F[:nF.value].copy(), xptr, xidx[:xptr[-1]].copy()


def kz_precode(plan: Plan, s, nrhs, xi, algo, sel, tol, max_iter, seed, x, v, iters, resid, status=None,
               rhs_per_cta=0, refresh=0, stream=None):
    lib = load()
    _check_c64(s, (nrhs, plan.K), "s")
    _check_c64(x, (nrhs, plan.Nt), "x")
    if v is not None:
        _check_c64(v, (nrhs, plan.K), "v")
    if iters.dtype != torch.int32 or resid.dtype != torch.float64:
        raise ValueError("iters must be int32 and resid float64")
    return _check(lib.kz_precode(plan.handle, _ptr(s), nrhs, float(xi), ALGOS[algo] if isinstance(algo, str) else algo,
                                 SELECT[sel] if isinstance(sel, str) else sel, float(tol), int(max_iter),
                                 int(seed), _ptr(x), _ptr(v), _ptr(iters), _ptr(resid), _ptr(status),
                                 int(rhs_per_cta), int(refresh), _stream(stream)))


def kz_precode_ex(plan: Plan, s, nrhs, xi, algo, sel, tol, max_iter, seed, x, v, iters, resid, status=None,
                  kernel="auto", rhs_per_cta=0, refresh=0, stream=None):
    lib = load()
    _check_c64(s, (nrhs, plan.K), "s")
    _check_c64(x, (nrhs, plan.Nt), "x")
    if v is not None:
        _check_c64(v, (nrhs, plan.K), "v")
    if iters.dtype != torch.int32 or resid.dtype != torch.float64:
        raise ValueError("iters must be int32 and resid float64")
    return _check(lib.kz_precode_ex(plan.handle, _ptr(s), nrhs, float(xi),
                                    ALGOS[algo] if isinstance(algo, str) else algo,
                                    SELECT[sel] if isinstance(sel, str) else sel, float(tol), int(max_iter),
                                    int(seed), _ptr(x), _ptr(v), _ptr(iters), _ptr(resid), _ptr(status),
                                    KERNELS[kernel] if isinstance(kernel, str) else kernel, int(rhs_per_cta),
                                    int(refresh), _stream(stream)))


class Batch:
    def __init__(self, handle, keep):
        self.handle = handle
        self.keep = keep  # the plans and tensors the device table points at
        self.nrhs = 0

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.kz_batch_destroy(self.handle)
            self.handle = None


def _batch_items(items, nrhs):
    arr = (KzBatchItem * len(items))()
    for k, it in enumerate(items):
        p = it["plan"]
        _check_c64(it["s"], (nrhs, p.K), "s")
        _check_c64(it["x"], (nrhs, p.Nt), "x")
        arr[k] = KzBatchItem(p.handle.value, it["s"].data_ptr(), it["x"].data_ptr(),
                             it["v"].data_ptr() if it.get("v") is not None else None, it["iters"].data_ptr(),
                             it["resid"].data_ptr(), float(it["xi"]))
    return arr


def kz_batch_prepare(items, nrhs, algo, prec="c64", rhs_per_cta=0, stream=None) -> Batch:
    """``items``: list of dicts with plan, s, x, v (or None), iters, resid, xi."""
    lib = load()
    arr = _batch_items(items, nrhs)
    h = ctypes.c_void_p()
    _check(lib.kz_batch_prepare(ctypes.byref(h), ctypes.cast(arr, ctypes.c_void_p), len(items), nrhs,
                                ALGOS[algo] if isinstance(algo, str) else algo, PREC[prec], int(rhs_per_cta),
                                _stream(stream)))
    b = Batch(h, list(items))
    b.nrhs = nrhs
    return b


def kz_batch_rebind(batch: Batch, items, stream=None):
    """Point the batch's items at new buffers / xi (same plans, same order)."""
    lib = load()
    if len(items) != len(batch.keep):
        raise ValueError("kz_batch_rebind: the batch has %d items" % len(batch.keep))
    arr = _batch_items(items, batch.nrhs)
    _check(lib.kz_batch_rebind(batch.handle, ctypes.cast(arr, ctypes.c_void_p), _stream(stream)))
    batch.keep = list(items)


def kz_batch_update(batch: Batch, H_cat, stream=None):
    """Re-pack every item's plan from H_cat (complex64 CUDA tensor: the items'
    packed channels concatenated in item order)."""
    lib = load()
    n = sum(it["plan"].sum_len for it in batch.keep)
    _check_c64(H_cat, (n,), "H_cat")
    return _check(lib.kz_batch_update(batch.handle, _ptr(H_cat), _stream(stream)))


def kz_batch_update_items(batch: Batch, H_cat, first, count, stream=None):
    """kz_batch_update for items [first, first + count): H_cat holds every
    item's packed channel in item order; only the range's are read."""
    lib = load()
    n = sum(it["plan"].sum_len for it in batch.keep)
    _check_c64(H_cat, (n,), "H_cat")
    return _check(lib.kz_batch_update_items(batch.handle, _ptr(H_cat), int(first), int(count), _stream(stream)))


def kz_precode_batched(batch: Batch, sel, tol, max_iter, seed, refresh=0, status=None, stream=None):
    lib = load()
    return _check(lib.kz_precode_batched(batch.handle, SELECT[sel] if isinstance(sel, str) else sel, float(tol),
                                         int(max_iter), int(seed), int(refresh), _ptr(status), _stream(stream)))


def kz_batch_tune(batch: Batch, sel, tol, max_iter, seed, stream=None):
    """Time the feasible launches on the batch; keep the fastest.
    Returns (kernel name, columns per CTA, threads)."""
    lib = load()
    chosen = np.zeros(3, dtype=np.int32)
    _check(lib.kz_batch_tune(batch.handle, SELECT[sel] if isinstance(sel, str) else sel, float(tol), int(max_iter),
                             int(seed), chosen.ctypes.data_as(ctypes.c_void_p), _stream(stream)))
    names = {v: k for k, v in KERNELS.items()}
    return names[int(chosen[0])], int(chosen[1]), int(chosen[2])


def kz_batch_query(batch: Batch):
    """The batch's launch: dict(kernel, rhs_per_cta, threads, launches)."""
    lib = load()
    v = [ctypes.c_int32() for _ in range(4)]
    _check(lib.kz_batch_query(batch.handle, *[ctypes.byref(x) for x in v]))
    names = {k: n for n, k in KERNELS.items()}
    return {"kernel": names.get(v[0].value, v[0].value), "rhs_per_cta": v[1].value, "threads": v[2].value,
            "launches": v[3].value}


def kz_batch_set_launch(batch: Batch, kernel, rhs_per_cta, threads, stream=None):
    lib = load()
    return _check(lib.kz_batch_set_launch(batch.handle, KERNELS[kernel] if isinstance(kernel, str) else kernel,
                                          int(rhs_per_cta), int(threads), _stream(stream)))


def kz_precode_adjoint(plan: Plan, nrhs, xi, Q, X, G_Q, G_X, tol, max_iter, lam, y, grad_H_packed, grad_xi, iters,
                       resid, status=None, stream=None):
    lib = load()
    return _check(lib.kz_precode_adjoint(plan.handle, nrhs, float(xi), _ptr(Q), _ptr(X), _ptr(G_Q), _ptr(G_X),
                                         float(tol), int(max_iter), _ptr(lam), _ptr(y), _ptr(grad_H_packed),
                                         _ptr(grad_xi), _ptr(iters), _ptr(resid), _ptr(status), _stream(stream)))


def kz_precode_adjoint_noalloc(plan: Plan, nrhs, xi, Q, X, G_Q, G_X, tol, max_iter, lam, y, grad_H_packed, grad_xi,
                               iters, resid, status=None, stream=None):
    """The adjoint without device allocation (for callers that cannot allocate
    when they differentiate, e.g. a real-time loop or a process whose device
    memory is reserved by another allocator); its scratch is a fixed 2 MiB
    device array shared by all calls on a device, so K * nrhs <= 262144."""
    lib = load()
    return _check(lib.kz_precode_adjoint_noalloc(plan.handle, nrhs, float(xi), _ptr(Q), _ptr(X), _ptr(G_Q),
                                                 _ptr(G_X), float(tol), int(max_iter), _ptr(lam), _ptr(y),
                                                 _ptr(grad_H_packed), _ptr(grad_xi), _ptr(iters), _ptr(resid),
                                                 _ptr(status), _stream(stream)))


def kz_precode_adjoint_batched(batch: Batch, items, tol, max_iter, status=None, stream=None):
    """``items``: list of dicts with Q, X, G_Q (or None), G_X (or None), grad_H, grad_xi."""
    lib = load()
    arr = (KzAdjointItem * len(items))()
    for k, it in enumerate(items):
        arr[k] = KzAdjointItem(it["Q"].data_ptr(), it["X"].data_ptr(),
                               it["G_Q"].data_ptr() if it.get("G_Q") is not None else None,
                               it["G_X"].data_ptr() if it.get("G_X") is not None else None,
                               it["grad_H"].data_ptr(), it["grad_xi"].data_ptr())
    return _check(lib.kz_precode_adjoint_batched(batch.handle, ctypes.cast(arr, ctypes.c_void_p), float(tol),
                                                 int(max_iter), _ptr(status), _stream(stream)))


def kz_precoder_matrix(plan: Plan, V, S, F, normalise=False, beta=None, stream=None):
    """F (ncols, Nt) from V (ncols, K) by the subarray form over S subarrays
    (both complex64 CUDA tensors, one row per column); beta: float32 (1,)."""
    lib = load()
    ncols = V.shape[0]
    _check_c64(V, (ncols, plan.K), "V")
    _check_c64(F, (ncols, plan.Nt), "F")
    if beta is not None and (beta.dtype != torch.float32 or tuple(beta.shape) != (1,)):
        raise ValueError("beta: expected float32 tensor of shape (1,)")
    return _check(lib.kz_precoder_matrix(plan.handle, _ptr(V), int(ncols), int(S), int(bool(normalise)), _ptr(F),
                                         _ptr(beta), _stream(stream)))


def kz_precode_record(plan: Plan, s, nrhs, xi, algo, sel, T, seed, x, v, iters, resid, hist_row, hist_gam,
                      status=None, stream=None):
    """T row projections per column with the selected-row history: hist_row
    int32 (T, nrhs), hist_gam complex64 (T, nrhs)."""
    lib = load()
    _check_c64(s, (nrhs, plan.K), "s")
    _check_c64(x, (nrhs, plan.Nt), "x")
    _check_c64(v, (nrhs, plan.K), "v")
    _check_c64(hist_gam, (T, nrhs), "hist_gam")
    if hist_row.dtype != torch.int32 or tuple(hist_row.shape) != (T, nrhs):
        raise ValueError("hist_row: expected int32 tensor of shape (T, nrhs)")
    return _check(lib.kz_precode_record(plan.handle, _ptr(s), int(nrhs), float(xi),
                                        ALGOS[algo] if isinstance(algo, str) else algo,
                                        SELECT[sel] if isinstance(sel, str) else sel, int(T), int(seed), _ptr(x),
                                        _ptr(v), _ptr(iters), _ptr(resid), _ptr(hist_row), _ptr(hist_gam),
                                        _ptr(status), _stream(stream)))


def kz_unrolled_adjoint(plan: Plan, nrhs, xi, T, iters, hist_row, hist_gam, x, v, G_X, G_V, grad_H, grad_xi, grad_s,
                        stream=None):
    lib = load()
    return _check(lib.kz_unrolled_adjoint(plan.handle, int(nrhs), float(xi), int(T), _ptr(iters), _ptr(hist_row),
                                          _ptr(hist_gam), _ptr(x), _ptr(v), _ptr(G_X), _ptr(G_V), _ptr(grad_H),
                                          _ptr(grad_xi), _ptr(grad_s), _stream(stream)))


def kz_plan_flops(plan: Plan, scheme, S, T):
    """Table I's FLOPs for the plan: scheme "rzf" or a method name (urk is rk_uniform)."""
    lib = load()
    code = -1 if scheme == "rzf" else (ALGOS["rk_uniform"] if scheme == "urk" else ALGOS[scheme])
    out = ctypes.c_double()
    _check(lib.kz_plan_flops(plan.handle, code, int(S), float(T), ctypes.byref(out)))
    return out.value


def kz_sum_rate(plan: Plan, X, snr_lin, sinr=None, rate=None, stream=None):
    """X: complex64 (K, Nt) (row k = user k's precoder column); sinr: float64 (K,); rate: float64 (1,)."""
    lib = load()
    _check_c64(X, (plan.K, plan.Nt), "X")
    for t, shape, name in ((sinr, (plan.K,), "sinr"), (rate, (1,), "rate")):
        if t is not None and (t.dtype != torch.float64 or tuple(t.shape) != shape):
            raise ValueError(f"{name}: expected float64 tensor of shape {shape}")
    return _check(lib.kz_sum_rate(plan.handle, _ptr(X), float(snr_lin), _ptr(sinr), _ptr(rate), _stream(stream)))


def kz_sum_rate_batched(batch: Batch, snr_lin, sinr=None, rate=None, stream=None):
    """sinr: float64 (n, K_max); rate: float64 (n,)."""
    lib = load()
    return _check(lib.kz_sum_rate_batched(batch.handle, float(snr_lin), _ptr(sinr), _ptr(rate), _stream(stream)))


def kz_version() -> int:
    return load().kz_version()


def exported_symbols():
    """Names of EXPORTS that the loaded library resolves."""
    lib = load()
    return [n for n in EXPORTS if hasattr(lib, n)]


# ----------------------------------------------------------------- convenience
def precode(plan: Plan, S, xi, algo="vr_oahk", sel="paper", tol=1e-6, max_iter=1000, seed=0, rhs_per_cta=0,
            refresh=0, want_v=True, sync=True, kernel="auto"):
    """Allocate outputs, run ``kz_precode`` and (by default) wait for it.

    ``S`` is a torch CUDA complex64 tensor of shape (nrhs, K).  Returns a dict
    with x (nrhs, Nt), v (nrhs, K), iters, resid and the status word.
    """
    nrhs = S.shape[0]
    dev = S.device
    x = torch.empty((nrhs, plan.Nt), dtype=torch.complex64, device=dev)
    v = torch.empty((nrhs, plan.K), dtype=torch.complex64, device=dev) if want_v else None
    iters = torch.empty(nrhs, dtype=torch.int32, device=dev)
    resid = torch.empty(nrhs, dtype=torch.float64, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    kz_precode_ex(plan, S, nrhs, xi, algo, sel, tol, max_iter, seed, x, v, iters, resid, status, kernel, rhs_per_cta,
                  refresh)
    out = {"x": x, "v": v, "iters": iters, "resid": resid, "status": status}
    if sync:
        torch.cuda.synchronize(dev)
        st = int(status.item())
        if st & KZ_STATUS_BIT_TIMEOUT:
            raise KzError(KZ_ERR_CUDA, "a bounded device wait expired")
        if st & KZ_STATUS_BIT_NUMERIC:
            raise KzError(KZ_ERR_NUMERIC, "NaN or Inf in a residual")
        out["converged"] = not (st & KZ_STATUS_BIT_NOT_CONVERGED)
    return out


def plan_from_instance(inst, prec="c64", device="cuda"):
    """Upload a ``kzgen.Instance``'s packed channel and build its plan."""
    Hp = torch.from_numpy(np.ascontiguousarray(inst.H_packed)).to(device)
    return kz_plan_create(inst.K, inst.Nt, inst.vr_offset, inst.vr_len, Hp, prec=prec)


def rhs_tensor(S_np, device="cuda"):
    """A K x nrhs NumPy matrix as the (nrhs, K) column-major device layout."""
    return torch.from_numpy(np.ascontiguousarray(np.asarray(S_np, dtype=np.complex64).T)).to(device)
