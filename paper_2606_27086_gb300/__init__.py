"""Python binding of the GB300 superiorized hyperslab-projection library.

Thin ctypes marshalling over the C ABI of ``include/suppy.h`` (the function
names are the same); every step of the method runs in the CUDA kernels of
``libsuppy_gb300.so``.  There is no CPU fallback: importing a function that
needs the library raises when the library has not been built.

Arrays may be numpy arrays (host) or torch CUDA tensors (device); one create
call takes all its arrays from one side.  PyTorch is used only for device
memory and streams.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# SUPPY_LIBRARY selects another build (e.g. libsuppy_gb300_checked.so)
LIB_PATH = os.environ.get("SUPPY_LIBRARY") or os.path.join(_HERE, "libsuppy_gb300.so")

SUPPY_OK, SUPPY_EINVAL, SUPPY_ENOMEM, SUPPY_ECUDA, SUPPY_ETIMEOUT, SUPPY_ESTATE = 0, -1, -2, -3, -4, -5
SUPPY_F32, SUPPY_BF16, SUPPY_F16, SUPPY_HALF_AUTO = 0, 1, 2, 3
SUPPY_CIMMINO, SUPPY_BIP, SUPPY_DROP, SUPPY_EL, SUPPY_EMR = 0, 1, 2, 3, 4
SUPPY_OBJ_NONE, SUPPY_OBJ_TV_ISO, SUPPY_OBJ_TV_ANISO, SUPPY_OBJ_LINEAR = 0, 1, 2, 3
SUPPY_OBJ_L1, SUPPY_OBJ_L2 = 4, 5
STRATEGY_AUTO, STRATEGY_ONE_PASS, STRATEGY_TWO_PASS, STRATEGY_TILED = 0, 1, 2, 3
SUPPY_DVC_UPPER, SUPPY_DVC_LOWER = 0, 1

EXPORTED = [
    "suppy_params_default", "suppy_create", "suppy_destroy", "suppy_set_stream",
    "suppy_set_bounds", "suppy_update_bounds", "suppy_update_bounds_async", "suppy_set_x", "suppy_get_x", "suppy_perturb",
    "suppy_sweep",
    "suppy_proximity", "suppy_objective", "suppy_run", "suppy_history", "suppy_get_state",
    "suppy_set_state", "suppy_info_get", "suppy_timing_enable", "suppy_kernel_time",
    "suppy_launch_count", "suppy_last_error", "suppy_version", "suppy_sweep_static",
    "suppy_server_create", "suppy_server_destroy", "suppy_server_add_matrix",
    "suppy_server_submit", "suppy_server_step", "suppy_server_query", "suppy_server_clock",
    "suppy_server_device_bytes", "suppy_server_last_error", "suppy_set_dvc", "suppy_dvc_dose",
    "suppy_dvc_proximity", "suppy_set_wait_limit",
]


class suppy_csr(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("n", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("val", ctypes.c_void_p),
                ("on_device", ctypes.c_int32)]


class suppy_opts(ctypes.Structure):
    _fields_ = [("a_dtype", ctypes.c_int), ("mode", ctypes.c_int),
                ("block_of_row", ctypes.c_void_p), ("nblocks", ctypes.c_int32),
                ("obj", ctypes.c_int), ("img_h", ctypes.c_int32), ("img_w", ctypes.c_int32),
                ("c_lin", ctypes.c_void_p), ("obj_rows", ctypes.POINTER(suppy_csr)),
                ("nrhs", ctypes.c_int32), ("box_len", ctypes.c_int64), ("tune", ctypes.c_int32),
                ("strategy", ctypes.c_int32), ("tma", ctypes.c_int32),
                ("stream_tile", ctypes.c_int32), ("stream_stages", ctypes.c_int32),
                ("stream_lanes", ctypes.c_int32), ("perturb_path", ctypes.c_int32),
                ("stream_map", ctypes.c_int32), ("tile_warps1", ctypes.c_int32),
                ("tile_chunk_bytes", ctypes.c_int32), ("tile_ring_bytes", ctypes.c_int32),
                ("tile_group_rows", ctypes.c_int32), ("stream_col_map", ctypes.c_int32),
                ("scatter_transpose", ctypes.c_int32)]


class suppy_params(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("gamma", ctypes.c_double),
                ("alpha", ctypes.c_double), ("n_red", ctypes.c_int32),
                ("max_trials", ctypes.c_int32), ("restart_every", ctypes.c_int32),
                ("max_sweeps", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("prox_abs", ctypes.c_double), ("prox_rel", ctypes.c_double),
                ("obj_rel", ctypes.c_double), ("patience", ctypes.c_int32),
                ("use_stopping", ctypes.c_int32), ("use_graphs", ctypes.c_int32),
                ("variance_tol", ctypes.c_double), ("adaptive", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("f_ref", ctypes.c_double)]


class suppy_stats(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int32), ("accepted", ctypes.c_int32),
                ("trials", ctypes.c_int32), ("stopped", ctypes.c_int32),
                ("ell", ctypes.c_int64), ("proximity", ctypes.c_double),
                ("objective", ctypes.c_double)]


class suppy_dvc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("structure", ctypes.c_int32),
                ("volume", ctypes.c_double), ("d_ref", ctypes.c_double)]


class suppy_server_opts(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_int64), ("slots", ctypes.c_int32),
                ("check_every", ctypes.c_int32)]


class suppy_request_info(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("sweeps", ctypes.c_int32),
                ("accepted", ctypes.c_int32), ("trials", ctypes.c_int32),
                ("proximity", ctypes.c_double), ("objective", ctypes.c_double),
                ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double),
                ("t_done", ctypes.c_double)]


class suppy_info(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("n", ctypes.c_int32), ("nrhs", ctypes.c_int32),
                ("m_kept", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("nnz_csc", ctypes.c_int64), ("nblocks", ctypes.c_int32),
                ("lanes_per_row", ctypes.c_int32), ("elems_in_regs", ctypes.c_int32),
                ("grid", ctypes.c_int32), ("block", ctypes.c_int32),
                ("perturb_cluster", ctypes.c_int32), ("device_bytes", ctypes.c_int64),
                ("strategy", ctypes.c_int32), ("scatter", ctypes.c_int32),
                ("col_lanes", ctypes.c_int32), ("col_grid", ctypes.c_int32),
                ("tma", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("stages", ctypes.c_int32), ("col_tile", ctypes.c_int32),
                ("col_stages", ctypes.c_int32), ("map", ctypes.c_int32),
                ("col_map", ctypes.c_int32), ("tiles", ctypes.c_int32),
                ("chunks", ctypes.c_int32), ("tile_warps1", ctypes.c_int32),
                ("tile_warps2", ctypes.c_int32), ("tile_coef_warps", ctypes.c_int32),
                ("tile_ring", ctypes.c_int32), ("tile_stream_bytes", ctypes.c_int64),
                ("tile_segments", ctypes.c_int64), ("transposed_rows", ctypes.c_int64),
                ("a_dtype", ctypes.c_int32), ("scatter_patch", ctypes.c_int32)]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the CUDA library (raises when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2606_27086_gb300.build.build()"
                           " -- there is no CPU fallback")
    lib = ctypes.CDLL(path)
    P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "suppy_params_default": (None, [ctypes.POINTER(suppy_params)]),
        "suppy_create": (ctypes.c_int, [ctypes.POINTER(suppy_csr), P, P, P, P,
                                        ctypes.POINTER(suppy_opts), P, ctypes.POINTER(P)]),
        "suppy_destroy": (None, [P]),
        "suppy_set_stream": (ctypes.c_int, [P, P]),
        "suppy_set_bounds": (ctypes.c_int, [P, P, P, I32]),
        "suppy_update_bounds": (ctypes.c_int, [P, P, P, I32]),
        "suppy_update_bounds_async": (ctypes.c_int, [P, P, P, I32]),
        "suppy_set_x": (ctypes.c_int, [P, P, I32]),
        "suppy_get_x": (ctypes.c_int, [P, P, I32]),
        "suppy_perturb": (ctypes.c_int, [P, ctypes.POINTER(suppy_params), P]),
        "suppy_sweep": (ctypes.c_int, [P, ctypes.POINTER(suppy_params), I32]),
        "suppy_proximity": (ctypes.c_int, [P, P]),
        "suppy_objective": (ctypes.c_int, [P, P]),
        "suppy_run": (ctypes.c_int, [P, ctypes.POINTER(suppy_params), P]),
        "suppy_history": (ctypes.c_int, [P, I32, P, P, I32, ctypes.POINTER(I32)]),
        "suppy_get_state": (ctypes.c_int, [P, P, ctypes.POINTER(ctypes.c_size_t)]),
        "suppy_set_state": (ctypes.c_int, [P, P, ctypes.c_size_t]),
        "suppy_info_get": (ctypes.c_int, [P, ctypes.POINTER(suppy_info)]),
        "suppy_timing_enable": (ctypes.c_int, [P, I32]),
        "suppy_kernel_time": (ctypes.c_int, [P, I32, ctypes.POINTER(D), ctypes.POINTER(I64)]),
        "suppy_launch_count": (I64, [P]),
        "suppy_last_error": (ctypes.c_char_p, [P]),
        "suppy_version": (ctypes.c_char_p, []),
        "suppy_sweep_static": (ctypes.c_int, [ctypes.POINTER(suppy_csr), P, P, ctypes.c_float,
                                              ctypes.c_float, P, P, I64, P, P, P]),
        "suppy_server_create": (ctypes.c_int, [ctypes.POINTER(suppy_server_opts), P]),
        "suppy_server_destroy": (None, [P]),
        "suppy_server_add_matrix": (ctypes.c_int, [P, ctypes.POINTER(suppy_csr), P, P,
                                                   ctypes.POINTER(suppy_opts),
                                                   ctypes.POINTER(suppy_params), P]),
        "suppy_server_submit": (ctypes.c_int, [P, I32, P, P, P]),
        "suppy_server_step": (ctypes.c_int, [P, P, P]),
        "suppy_server_query": (ctypes.c_int, [P, I64, ctypes.POINTER(suppy_request_info), P]),
        "suppy_server_clock": (D, [P]),
        "suppy_server_device_bytes": (I64, [P]),
        "suppy_server_last_error": (ctypes.c_char_p, [P]),
        "suppy_set_dvc": (ctypes.c_int, [P, ctypes.POINTER(suppy_csr), P, I32,
                                         ctypes.POINTER(suppy_dvc), I32, D]),
        "suppy_dvc_dose": (ctypes.c_int, [P, P, I32]),
        "suppy_dvc_proximity": (ctypes.c_int, [P, P]),
        "suppy_set_wait_limit": (ctypes.c_int, [P, I64]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class SuppyError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"suppy status {status}: {msg}")
        self.status = status


def _check(status: int, ctx) -> None:
    if status != SUPPY_OK:
        msg = load_library().suppy_last_error(ctx)
        raise SuppyError(status, msg.decode() if msg else "")


def _ptr(a):
    """(pointer, on_device, keepalive) of a numpy array or torch tensor."""
    if a is None:
        return None, 0, None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            a = a.contiguous()
        return ctypes.c_void_p(a.data_ptr()), int(a.is_cuda), a
    arr = np.ascontiguousarray(a)
    return ctypes.c_void_p(arr.ctypes.data), 0, arr


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def suppy_params_default(**overrides) -> suppy_params:
    p = suppy_params()
    load_library().suppy_params_default(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, "lambda_" if k in ("lam", "lambda") else k, v)
    return p


def _csr(row_ptr, col, val, m, n, keep):
    rp, d1, k1 = _ptr(row_ptr)
    cp, d2, k2 = _ptr(col)
    vp, d3, k3 = _ptr(val)
    keep += [k1, k2, k3]
    if not (d1 == d2 == d3):
        raise ValueError("row_ptr, col and val must live on the same side")
    nnz = int(val.shape[0]) if hasattr(val, "shape") else len(val)
    return suppy_csr(int(m), int(n), nnz, rp, cp, vp, d1)


class Context:
    """Owns one ``suppy_ctx``; methods call the C ABI functions of the same name."""

    def __init__(self, row_ptr, col, val, m, n, l, u, box_lo, box_hi, *, dtype=SUPPY_F32,
                 mode=SUPPY_CIMMINO, block_of_row=None, obj=SUPPY_OBJ_NONE, shape=None,
                 c_lin=None, obj_rows=None, nrhs=1, tune=0, strategy=0, tma=0, stream=None,
                 stream_shape=(0, 0, 0), perturb_path=0, stream_map=0, tile_warps1=0,
                 tile_chunk_bytes=0, tile_ring_bytes=0, tile_group_rows=0, stream_col_map=0,
                 scatter_transpose=0):
        lib = load_library()
        self._lib = lib
        keep = []
        A = _csr(row_ptr, col, val, m, n, keep)
        lp, dl, kl = _ptr(l)
        up, du, ku = _ptr(u)
        lop, _, klo = _ptr(box_lo)
        hip, _, khi = _ptr(box_hi)
        keep += [kl, ku, klo, khi]
        o = suppy_opts()
        o.a_dtype = dtype
        o.mode = mode
        if block_of_row is not None:
            bor = np.ascontiguousarray(np.asarray(block_of_row), dtype=np.int32)
            keep.append(bor)
            o.block_of_row = ctypes.c_void_p(bor.ctypes.data)
            o.nblocks = int(bor.max()) + 1 if bor.size else 1
        o.obj = obj
        if shape is not None:
            o.img_h, o.img_w = int(shape[0]), int(shape[1])
        if c_lin is not None:
            cp, _, kc = _ptr(c_lin)
            keep.append(kc)
            o.c_lin = cp
        if obj_rows is not None:
            S = _csr(*obj_rows, keep=keep) if isinstance(obj_rows, tuple) else obj_rows
            keep.append(S)
            o.obj_rows = ctypes.pointer(S)
        o.nrhs = int(nrhs)
        blen = box_lo.shape[0] if hasattr(box_lo, "shape") else len(box_lo)
        o.box_len = int(blen)
        o.tune = int(tune)
        o.strategy = int(strategy)
        o.tma = int(tma)
        o.stream_tile, o.stream_stages, o.stream_lanes = (int(v) for v in stream_shape)
        o.perturb_path = int(perturb_path)
        o.stream_map = int(stream_map)
        o.tile_warps1 = int(tile_warps1)
        o.tile_chunk_bytes = int(tile_chunk_bytes)
        o.tile_ring_bytes = int(tile_ring_bytes)
        o.tile_group_rows = int(tile_group_rows)
        o.stream_col_map = int(stream_col_map)
        o.scatter_transpose = int(scatter_transpose)
        ctx = ctypes.c_void_p()
        self._keep = keep
        self.m, self.n, self.nrhs = int(m), int(n), int(nrhs)
        self.mq = 0                 # rows of the dose-volume matrix (suppy_set_dvc)
        st = lib.suppy_create(ctypes.byref(A), lp, up, lop, hip, ctypes.byref(o),
                              _stream_handle(stream), ctypes.byref(ctx))
        _check(st, None)
        self.ctx = ctx
        self._keep = None

    # -- lifetime
    def close(self):
        if getattr(self, "ctx", None):
            self._lib.suppy_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- C ABI wrappers (same names)
    def suppy_set_stream(self, stream):
        _check(self._lib.suppy_set_stream(self.ctx, _stream_handle(stream)), self.ctx)

    def suppy_set_bounds(self, l, u):
        lp, dl, k1 = _ptr(l)
        up, du, k2 = _ptr(u)
        _check(self._lib.suppy_set_bounds(self.ctx, lp, up, dl), self.ctx)

    def suppy_update_bounds(self, l, u):
        lp, dl, k1 = _ptr(l)
        up, du, k2 = _ptr(u)
        _check(self._lib.suppy_update_bounds(self.ctx, lp, up, dl), self.ctx)

    def suppy_update_bounds_async(self, l, u):
        """Enqueue-only bounds update; keep l and u alive and unchanged until the
        next synchronizing call (which reports a rejected set)."""
        lp, dl, k1 = _ptr(l)
        up, du, k2 = _ptr(u)
        self._pending_bounds = (k1, k2)
        _check(self._lib.suppy_update_bounds_async(self.ctx, lp, up, dl), self.ctx)

    def suppy_set_x(self, x):
        xp, d, k = _ptr(x)
        _check(self._lib.suppy_set_x(self.ctx, xp, d), self.ctx)

    def suppy_get_x(self, out=None):
        if out is None:
            out = np.empty((self.n, self.nrhs) if self.nrhs > 1 else self.n, dtype=np.float32)
        xp, d, k = _ptr(out)
        _check(self._lib.suppy_get_x(self.ctx, xp, d), self.ctx)
        return out

    def suppy_perturb(self, params: suppy_params, want_accepted: bool = True):
        acc = np.zeros(self.nrhs, dtype=np.int32) if want_accepted else None
        ap = ctypes.c_void_p(acc.ctypes.data) if acc is not None else None
        _check(self._lib.suppy_perturb(self.ctx, ctypes.byref(params), ap), self.ctx)
        return acc

    def suppy_sweep(self, params: suppy_params, nsweeps: int = 1):
        _check(self._lib.suppy_sweep(self.ctx, ctypes.byref(params), int(nsweeps)), self.ctx)

    def suppy_proximity(self):
        out = np.zeros(self.nrhs, dtype=np.float64)
        _check(self._lib.suppy_proximity(self.ctx, ctypes.c_void_p(out.ctypes.data)), self.ctx)
        return out

    def suppy_set_dvc(self, row_ptr, col, val, m, structure_ptr, dvcs, relax: float = 1.0):
        """dvcs: sequence of (kind, structure, volume, d_ref); empty removes the sets."""
        if not len(dvcs):
            _check(self._lib.suppy_set_dvc(self.ctx, None, None, 0, None, 0, float(relax)),
                   self.ctx)
            self.mq = 0
            return
        keep = []
        A = _csr(row_ptr, col, val, m, self.n, keep)
        sp = np.ascontiguousarray(structure_ptr, dtype=np.int32)
        arr = (suppy_dvc * max(len(dvcs), 1))()
        for j, (kind, st, vol, dref) in enumerate(dvcs):
            arr[j] = suppy_dvc(int(kind), int(st), float(vol), float(dref))
        _check(self._lib.suppy_set_dvc(self.ctx, ctypes.byref(A), ctypes.c_void_p(sp.ctypes.data),
                                       len(sp) - 1, arr, len(dvcs), float(relax)), self.ctx)
        self.mq = int(m) if len(dvcs) else 0

    def suppy_dvc_dose(self, out=None):
        """Doses A_q x: m_q values, or m_q x B for several right-hand sides."""
        if out is None:
            shape = (self.mq,) if self.nrhs == 1 else (self.mq, self.nrhs)
            out = np.empty(shape, dtype=np.float32)
        op, d, k = _ptr(out)
        _check(self._lib.suppy_dvc_dose(self.ctx, op, d), self.ctx)
        return out

    def suppy_dvc_proximity(self):
        """Target-space proximity: a float, or B values for several right-hand sides."""
        v = np.zeros(max(1, self.nrhs), dtype=np.float64)
        _check(self._lib.suppy_dvc_proximity(self.ctx, ctypes.c_void_p(v.ctypes.data)), self.ctx)
        return float(v[0]) if self.nrhs == 1 else v

    def suppy_objective(self):
        out = np.zeros(self.nrhs, dtype=np.float64)
        _check(self._lib.suppy_objective(self.ctx, ctypes.c_void_p(out.ctypes.data)), self.ctx)
        return out

    def suppy_run(self, params: suppy_params, want_stats: bool = True):
        """With want_stats False (and params.use_stopping 0) the call only
        enqueues the iterations and returns None."""
        if not want_stats:
            _check(self._lib.suppy_run(self.ctx, ctypes.byref(params), None), self.ctx)
            return None
        st = (suppy_stats * self.nrhs)()
        _check(self._lib.suppy_run(self.ctx, ctypes.byref(params), ctypes.cast(st, ctypes.c_void_p)),
               self.ctx)
        return [dict(sweeps=s.sweeps, accepted=s.accepted, trials=s.trials, stopped=s.stopped,
                     ell=s.ell, proximity=s.proximity, objective=s.objective) for s in st]

    def suppy_history(self, rhs: int = 0, cap: int = 1 << 16):
        cnt = ctypes.c_int32()
        _check(self._lib.suppy_history(self.ctx, int(rhs), None, None, 0, ctypes.byref(cnt)),
               self.ctx)
        k = min(cnt.value, cap)
        prox = np.zeros(k, dtype=np.float64)
        obj = np.zeros(k, dtype=np.float64)
        _check(self._lib.suppy_history(self.ctx, int(rhs), ctypes.c_void_p(prox.ctypes.data),
                                       ctypes.c_void_p(obj.ctypes.data), k, ctypes.byref(cnt)),
               self.ctx)
        return prox, obj

    def suppy_get_state(self) -> bytes:
        ln = ctypes.c_size_t()
        _check(self._lib.suppy_get_state(self.ctx, None, ctypes.byref(ln)), self.ctx)
        buf = ctypes.create_string_buffer(ln.value)
        _check(self._lib.suppy_get_state(self.ctx, buf, ctypes.byref(ln)), self.ctx)
        return buf.raw

    def suppy_set_state(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(self._lib.suppy_set_state(self.ctx, buf, len(blob)), self.ctx)

    def suppy_info_get(self) -> dict:
        inf = suppy_info()
        _check(self._lib.suppy_info_get(self.ctx, ctypes.byref(inf)), self.ctx)
        return {k: getattr(inf, k) for k, _ in suppy_info._fields_}

    def suppy_set_wait_limit(self, cycles: int = 0):
        """Budget of every bounded device wait in SM cycles (0: the default)."""
        _check(self._lib.suppy_set_wait_limit(self.ctx, int(cycles)), self.ctx)

    def suppy_timing_enable(self, enable: bool = True):
        _check(self._lib.suppy_timing_enable(self.ctx, int(enable)), self.ctx)

    def suppy_kernel_time(self, kind: int = 0):
        """(total ms, launches) of kernel kind 0 row pass, 1 box step, 2 perturbation."""
        ms = ctypes.c_double()
        nl = ctypes.c_int64()
        _check(self._lib.suppy_kernel_time(self.ctx, int(kind), ctypes.byref(ms), ctypes.byref(nl)),
               self.ctx)
        return ms.value, nl.value

    def suppy_launch_count(self) -> int:
        return int(self._lib.suppy_launch_count(self.ctx))


def from_problem(prob, *, dtype=SUPPY_F32, mode=SUPPY_CIMMINO, obj=SUPPY_OBJ_NONE, device=False,
                 stream=None, tune=0, strategy=0, tma=0, stream_shape=(0, 0, 0),
                 perturb_path=0, stream_map=0, tile_warps1=0, tile_chunk_bytes=0,
                 tile_ring_bytes=0, tile_group_rows=0, stream_col_map=0,
                 scatter_transpose=0) -> Context:
    """Create a context from a ``synth.Problem`` (host arrays, or copied to the
    current CUDA device first when ``device`` is True)."""
    A = prob.A
    l, u = prob.l, prob.u
    nrhs = 1 if l.ndim == 1 else l.shape[1]
    arrs = [A.row_ptr, A.col, A.val, l, u, prob.box_lo, prob.box_hi]
    if device:
        import torch
        arrs = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]
    rp, col, val, l, u, lo, hi = arrs
    kw = {}
    # the image grid: required by the TV objectives, and where the tiled
    # sweep cuts its tiles with any objective
    if prob.shape is not None and len(prob.shape) == 2:
        kw["shape"] = prob.shape
    if obj == SUPPY_OBJ_LINEAR:
        if prob.body is not None:
            b = prob.body
            kw["obj_rows"] = (b.row_ptr, b.col, b.val, b.m, b.n)
        else:
            kw["c_lin"] = prob.c_lin
    blocks = prob.blocks if mode == SUPPY_BIP else None
    return Context(rp, col, val, A.m, A.n, l, u, lo, hi, dtype=dtype, mode=mode,
                   block_of_row=blocks, obj=obj, nrhs=nrhs, stream=stream, tune=tune,
                   strategy=strategy, tma=tma, stream_shape=stream_shape,
                   perturb_path=perturb_path, stream_map=stream_map, tile_warps1=tile_warps1,
                   tile_chunk_bytes=tile_chunk_bytes, tile_ring_bytes=tile_ring_bytes,
                   tile_group_rows=tile_group_rows, stream_col_map=stream_col_map,
                   scatter_transpose=scatter_transpose, **kw)


def suppy_sweep_static(row_ptr, col, val, m, n, l, u, weight, lam, box_lo, box_hi, x,
                       proximity=None, stream=None):
    """One allocation-free sweep on device tensors (see include/suppy.h);
    x is updated in place, proximity (a one-element float64 device tensor)
    receives the proximity of the input point."""
    lib = load_library()
    keep = []
    A = _csr(row_ptr, col, val, m, n, keep)
    args = [_ptr(t)[0] for t in (l, u, box_lo, box_hi, x)]
    bl = box_lo.shape[0] if hasattr(box_lo, "shape") else len(box_lo)
    pp = _ptr(proximity)[0] if proximity is not None else None
    st = lib.suppy_sweep_static(ctypes.byref(A), args[0], args[1], float(weight), float(lam),
                                args[2], args[3], int(bl), args[4], pp, _stream_handle(stream))
    _check(st, None)


def version() -> str:
    return load_library().suppy_version().decode()


class Server:
    """Owns one ``suppy_server`` (continuous batching of many solves); methods
    call the C ABI functions of the same name."""

    def __init__(self, hbm_budget: int = 0, slots: int = 32, check_every: int = 8):
        self._lib = load_library()
        o = suppy_server_opts(int(hbm_budget), int(slots), int(check_every))
        h = ctypes.c_void_p()
        st = self._lib.suppy_server_create(ctypes.byref(o), ctypes.byref(h))
        _check(st, None)
        self.srv = h
        self.matrices = []

    def _check(self, st):
        if st != SUPPY_OK:
            msg = self._lib.suppy_server_last_error(self.srv)
            raise SuppyError(st, msg.decode() if msg else "")

    def suppy_server_add_matrix(self, prob, params: suppy_params, *, dtype=SUPPY_F32,
                                mode=SUPPY_CIMMINO, obj=SUPPY_OBJ_NONE, strategy=0) -> int:
        """Register the matrix, box and objective of a ``synth.Problem``."""
        A = prob.A
        keep = []
        csr = _csr(A.row_ptr, A.col, A.val, A.m, A.n, keep)
        lop, _, k1 = _ptr(np.ascontiguousarray(prob.box_lo, np.float32))
        hip, _, k2 = _ptr(np.ascontiguousarray(prob.box_hi, np.float32))
        keep += [k1, k2]
        o = suppy_opts()
        o.a_dtype = dtype
        o.mode = mode
        if mode == SUPPY_BIP and prob.blocks is not None:
            bor = np.ascontiguousarray(prob.blocks, dtype=np.int32)
            keep.append(bor)
            o.block_of_row = ctypes.c_void_p(bor.ctypes.data)
            o.nblocks = int(bor.max()) + 1
        o.obj = obj
        if obj in (SUPPY_OBJ_TV_ISO, SUPPY_OBJ_TV_ANISO):
            o.img_h, o.img_w = int(prob.shape[0]), int(prob.shape[1])
        if obj == SUPPY_OBJ_LINEAR:
            if prob.body is not None:
                b = prob.body
                S = _csr(b.row_ptr, b.col, b.val, b.m, b.n, keep)
                keep.append(S)
                o.obj_rows = ctypes.pointer(S)
            else:
                cp, _, kc = _ptr(np.ascontiguousarray(prob.c_lin, np.float32))
                keep.append(kc)
                o.c_lin = cp
        o.box_len = int(np.asarray(prob.box_lo).shape[0])
        o.strategy = int(strategy)
        mid = ctypes.c_int32()
        self._check(self._lib.suppy_server_add_matrix(self.srv, ctypes.byref(csr), lop, hip,
                                                      ctypes.byref(o), ctypes.byref(params),
                                                      ctypes.byref(mid)))
        self.matrices.append((A.m, A.n))
        return mid.value

    def suppy_server_submit(self, matrix_id: int, l, u) -> int:
        l = np.ascontiguousarray(l, np.float32)
        u = np.ascontiguousarray(u, np.float32)
        rid = ctypes.c_int64()
        self._check(self._lib.suppy_server_submit(self.srv, int(matrix_id),
                                                  ctypes.c_void_p(l.ctypes.data),
                                                  ctypes.c_void_p(u.ctypes.data),
                                                  ctypes.byref(rid)))
        return rid.value

    def suppy_server_step(self):
        r, w = ctypes.c_int32(), ctypes.c_int32()
        self._check(self._lib.suppy_server_step(self.srv, ctypes.byref(r), ctypes.byref(w)))
        return r.value, w.value

    def suppy_server_query(self, request_id: int, n: int | None = None):
        info = suppy_request_info()
        x = np.zeros(n, np.float32) if n else None
        xp = ctypes.c_void_p(x.ctypes.data) if x is not None else None
        self._check(self._lib.suppy_server_query(self.srv, int(request_id), ctypes.byref(info),
                                                 xp))
        d = {k: getattr(info, k) for k, _ in suppy_request_info._fields_}
        return d, (x if d["state"] == 2 else None)

    def suppy_server_clock(self) -> float:
        return self._lib.suppy_server_clock(self.srv)

    def suppy_server_device_bytes(self) -> int:
        return self._lib.suppy_server_device_bytes(self.srv)

    def close(self):
        if getattr(self, "srv", None):
            self._lib.suppy_server_destroy(self.srv)
            self.srv = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
