"""GB300-native graph-coloured H^1 peeling compression (Levitt & Martinsson).

Thin ctypes binding of the C ABI in include/hm.h: the functions below carry the
C names and only marshal arguments; every step of the compression runs in the
CUDA kernels of libhm.so.  PyTorch provides device memory and streams.

If libhm.so has not been built this module raises ImportError: there is no
CPU fallback.  Build it with ``python -c "import __graft_entry__ as g; g.build()"``
(or ``python paper_2205_03406_gb300/_build.py``).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhm.so")

HM_OK, HM_EINVAL, HM_ENOMEM, HM_ESTATE, HM_ECUDA, HM_EOP, HM_ETIMEOUT, HM_ENOTSUP = range(8)
STATUS_NAMES = ["HM_OK", "HM_EINVAL", "HM_ENOMEM", "HM_ESTATE", "HM_ECUDA", "HM_EOP", "HM_ETIMEOUT",
                "HM_ENOTSUP"]
HM_FP64, HM_MIXED_BF16X6, HM_MIXED_BF16X6_F32 = 0, 1, 2
HM_FORMAT_H1, HM_FORMAT_UNIFORM_H1, HM_FORMAT_H2 = 0, 1, 2
HM_K_LOG, HM_K_LAPLACE3D, HM_K_INVR, HM_K_EXP = 1, 2, 3, 4
HM_OP_KERNEL, HM_OP_DENSE, HM_OP_CALLBACK = 0, 1, 2
HM_LEVEL_LEAF = -1
(HM_X_PERM, HM_X_LEVEL_BOXES, HM_X_CUT, HM_X_NEAR, HM_X_INTER, HM_X_PAIR_VERTEX, HM_X_VERTEX_COLOR,
 HM_X_VERTEX_BETA, HM_X_GAUSS, HM_X_SAMPLE_Y, HM_X_SAMPLE_Z, HM_X_PAIR_RANKS, HM_X_FACTORS,
 HM_X_FACTOR_OFFS, HM_X_LEAF_D, HM_X_VERTEX_DEGREE, HM_X_BOX_VERTEX_BOX, HM_X_BOX_COLOR,
 HM_X_BOX_DEGREE, HM_X_H2_RANKS, HM_X_H2_SIGMA) = range(1, 22)

EXPORTED = ["hm_create", "hm_destroy", "hm_tree_build", "hm_color", "hm_sample", "hm_compress", "hm_apply",
            "hm_relerr", "hm_get_info", "hm_export", "hm_last_error", "hm_apply_noalloc", "hm_color_boxes",
            "hm_server_create", "hm_server_submit", "hm_server_wait", "hm_server_apply", "hm_server_release",
            "hm_server_get_info", "hm_server_destroy"]
HM_JOB_QUEUED, HM_JOB_RUNNING, HM_JOB_READY, HM_JOB_FAILED = range(4)


class hm_config(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("leaf_size", ctypes.c_int), ("uniform_depth", ctypes.c_int),
                ("r", ctypes.c_int), ("oversample", ctypes.c_int), ("rank", ctypes.c_int),
                ("tol", ctypes.c_double),
                ("precision", ctypes.c_int), ("keep_samples", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("format", ctypes.c_int)]


HM_APPLY_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                               ctypes.c_int64, ctypes.c_void_p)


class hm_op(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("kernel", ctypes.c_int), ("dense_dev", ctypes.c_void_p),
                ("apply", HM_APPLY_FN), ("user", ctypes.c_void_p)]


class hm_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("L", ctypes.c_int), ("n_boxes", ctypes.c_int),
                ("colors", ctypes.c_int * 32), ("pairs", ctypes.c_int64 * 32), ("vertices", ctypes.c_int64 * 32),
                ("matvec_cols", ctypes.c_int64), ("factor_floats", ctypes.c_int64), ("max_rank", ctypes.c_int),
                ("seconds_sample", ctypes.c_double), ("seconds_total", ctypes.c_double),
                ("seconds_phase", ctypes.c_double * 8), ("act_rows", ctypes.c_int64 * 32),
                ("kernel_launches", ctypes.c_int64), ("launches_total", ctypes.c_int64),
                ("tc_kernel_evals", ctypes.c_int64), ("device_allocs", ctypes.c_int64),
                ("bb_tc_levels", ctypes.c_int), ("bb_fp64_levels", ctypes.c_int), ("leaf_size", ctypes.c_int),
                ("rank", ctypes.c_int), ("tol", ctypes.c_double), ("seconds_peel_update", ctypes.c_double),
                ("peel_update_macs", ctypes.c_int64), ("pool_used_bytes", ctypes.c_uint64),
                ("pool_peak_bytes", ctypes.c_uint64)]

class hm_server_config(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_size_t), ("slots", ctypes.c_int)]


class hm_job_desc(ctypes.Structure):
    _fields_ = [("cfg", hm_config), ("op", hm_op), ("points_host", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("leaf_size", ctypes.c_int), ("tol", ctypes.c_double), ("rank", ctypes.c_int)]


class hm_job_stats(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int), ("status", ctypes.c_int), ("t_submit", ctypes.c_double),
                ("t_start", ctypes.c_double), ("t_done", ctypes.c_double), ("reserved_bytes", ctypes.c_size_t),
                ("estimate_bytes", ctypes.c_size_t), ("info", hm_info)]


class hm_server_info(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("released", ctypes.c_int64), ("queued", ctypes.c_int64), ("running", ctypes.c_int64),
                ("max_running", ctypes.c_int), ("budget", ctypes.c_size_t), ("reserved", ctypes.c_size_t),
                ("max_reserved", ctypes.c_size_t), ("jobs_per_s", ctypes.c_double), ("job_p50_s", ctypes.c_double),
                ("job_p99_s", ctypes.c_double), ("applies", ctypes.c_int64), ("apply_p50_s", ctypes.c_double),
                ("apply_p99_s", ctypes.c_double)]


PHASES = ["colouring", "test matrices", "black box", "peel", "bases+cores", "leaf black box", "leaf peel+extract",
          "tensor-core kernel"]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first "
                          "(python -c 'import __graft_entry__ as g; g.build()'); there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    sig = {
        "hm_create": [ctypes.POINTER(P), ctypes.POINTER(hm_config), P],
        "hm_destroy": [P],
        "hm_tree_build": [P, P, I64, I],
        "hm_color": [P, I, ctypes.POINTER(I)],
        "hm_color_boxes": [P, I, ctypes.POINTER(I)],
        "hm_sample": [P, ctypes.POINTER(hm_op), I],
        "hm_compress": [P, ctypes.POINTER(hm_op), D, I],
        "hm_apply": [P, P, P, I64, I],
        "hm_apply_noalloc": [P, P, P, I64, I],
        "hm_relerr": [P, ctypes.POINTER(hm_op), I, ctypes.POINTER(D)],
        "hm_get_info": [P, ctypes.POINTER(hm_info)],
        "hm_export": [P, I, I, P, ctypes.POINTER(ctypes.c_size_t)],
        "hm_last_error": [P],
        "hm_server_create": [ctypes.POINTER(P), ctypes.POINTER(hm_server_config)],
        "hm_server_submit": [P, ctypes.POINTER(hm_job_desc), ctypes.POINTER(I64)],
        "hm_server_wait": [P, I64, D, ctypes.POINTER(hm_job_stats)],
        "hm_server_apply": [P, I64, P, P, I64, I],
        "hm_server_release": [P, I64],
        "hm_server_get_info": [P, ctypes.POINTER(hm_server_info)],
        "hm_server_destroy": [P],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_char_p if name == "hm_last_error" else ctypes.c_int
    return lib


_lib = _load()


class HMError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")


def lib():
    return _lib


def _check(ctx, st: int, where: str):
    if st != HM_OK:
        msg = _lib.hm_last_error(ctx).decode() if ctx else ""
        raise HMError(st, where, msg)


# ---------------------------------------------------------------------------
# functions with the C names (argument marshalling only)
# ---------------------------------------------------------------------------

def hm_create(cfg: hm_config, stream: int = 0):
    ctx = ctypes.c_void_p()
    _check(None, _lib.hm_create(ctypes.byref(ctx), ctypes.byref(cfg), ctypes.c_void_p(stream)), "hm_create")
    return ctx


def hm_destroy(ctx):
    return _lib.hm_destroy(ctx)


def hm_tree_build(ctx, points_dev: int, n: int, leaf_size: int = 0):
    _check(ctx, _lib.hm_tree_build(ctx, ctypes.c_void_p(points_dev), n, leaf_size), "hm_tree_build")


def hm_color(ctx, level: int) -> int:
    nc = ctypes.c_int(0)
    _check(ctx, _lib.hm_color(ctx, level, ctypes.byref(nc)), "hm_color")
    return nc.value


def hm_color_boxes(ctx, level: int) -> int:
    nc = ctypes.c_int(0)
    _check(ctx, _lib.hm_color_boxes(ctx, level, ctypes.byref(nc)), "hm_color_boxes")
    return nc.value


def hm_sample(ctx, op: hm_op, level: int):
    _check(ctx, _lib.hm_sample(ctx, ctypes.byref(op), level), "hm_sample")


def hm_compress(ctx, op: hm_op, tol: float = 0.0, rank: int = 0):
    _check(ctx, _lib.hm_compress(ctx, ctypes.byref(op), tol, rank), "hm_compress")


def hm_apply(ctx, x_dev: int, y_dev: int, nrhs: int, trans: int = 0):
    _check(ctx, _lib.hm_apply(ctx, ctypes.c_void_p(x_dev), ctypes.c_void_p(y_dev), nrhs, trans), "hm_apply")


def hm_apply_noalloc(ctx, x_dev: int, y_dev: int, nrhs: int, trans: int = 0):
    _check(ctx, _lib.hm_apply_noalloc(ctx, ctypes.c_void_p(x_dev), ctypes.c_void_p(y_dev), nrhs, trans),
           "hm_apply_noalloc")


def hm_relerr(ctx, op: hm_op, iters: int = 20) -> float:
    e = ctypes.c_double(0.0)
    _check(ctx, _lib.hm_relerr(ctx, ctypes.byref(op), iters, ctypes.byref(e)), "hm_relerr")
    return e.value


def hm_get_info(ctx) -> hm_info:
    info = hm_info()
    _check(ctx, _lib.hm_get_info(ctx, ctypes.byref(info)), "hm_get_info")
    return info


def hm_export(ctx, what: int, level: int = 0) -> bytes:
    size = ctypes.c_size_t(0)
    _check(ctx, _lib.hm_export(ctx, what, level, None, ctypes.byref(size)), "hm_export")
    buf = ctypes.create_string_buffer(max(size.value, 1))
    _check(ctx, _lib.hm_export(ctx, what, level, buf, ctypes.byref(size)), "hm_export")
    return buf.raw[:size.value]


def hm_export_into(ctx, what: int, level: int, host_ptr: int, nbytes: int) -> int:
    """hm_export into caller memory (host_ptr, nbytes); returns the bytes written."""
    size = ctypes.c_size_t(nbytes)
    _check(ctx, _lib.hm_export(ctx, what, level, ctypes.c_void_p(host_ptr), ctypes.byref(size)), "hm_export")
    return size.value


def hm_export_size(ctx, what: int, level: int = 0) -> int:
    size = ctypes.c_size_t(0)
    _check(ctx, _lib.hm_export(ctx, what, level, None, ctypes.byref(size)), "hm_export")
    return size.value


def hm_last_error(ctx) -> str:
    return _lib.hm_last_error(ctx).decode()


# ---------------------------------------------------------------------------
# convenience wrapper around torch device tensors
# ---------------------------------------------------------------------------

def kernel_op(kernel: int) -> hm_op:
    op = hm_op()
    op.kind = HM_OP_KERNEL
    op.kernel = kernel
    return op


def dense_op(a_dev) -> hm_op:
    """Stored dense operator; a_dev is a torch float64 CUDA tensor (n x n, row i = A[i, :]).
    The library reads it column-major, so pass A^T's storage: a contiguous tensor of A.T."""
    op = hm_op()
    op.kind = HM_OP_DENSE
    op.dense_dev = a_dev.data_ptr()
    op._keep = a_dev
    return op


def callback_op(fn) -> hm_op:
    """fn(trans, X_ptr, Y_ptr, s, stream) -> int: user black box on raw device pointers."""
    op = hm_op()
    op.kind = HM_OP_CALLBACK
    op.apply = HM_APPLY_FN(lambda user, trans, x, y, s, st: fn(trans, x, y, s, st))
    op._keep = op.apply
    return op


@dataclass
class Settings:
    d: int
    leaf_size: int = 64
    r: int = 32
    oversample: int = 10
    rank: int = 0
    tol: float = 0.0
    uniform_depth: int = 0
    precision: int = HM_FP64
    keep_samples: bool = False
    seed: int = 0
    format: int = HM_FORMAT_H1

    def to_c(self) -> hm_config:
        return hm_config(self.d, self.leaf_size, self.uniform_depth, self.r, self.oversample, self.rank,
                         self.tol, self.precision, int(self.keep_samples), self.seed, self.format)


class Compressor:
    """One compression job: owns an hm_ctx on a torch CUDA stream."""

    def __init__(self, settings: Settings, stream=None):
        import torch
        self.torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.settings = settings
        self.ctx = hm_create(settings.to_c(), self.stream.cuda_stream)

    def close(self):
        if self.ctx:
            hm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def tree_build(self, points, leaf_size: int = 0):
        """Cluster tree of the points (leaf_size 0: the settings' leaf size)."""
        pts = points.to(device="cuda", dtype=self.torch.float64).contiguous()
        self._points = pts
        hm_tree_build(self.ctx, pts.data_ptr(), pts.shape[0], leaf_size)
        return self

    def color(self, level: int) -> int:
        return hm_color(self.ctx, level)

    def color_boxes(self, level: int) -> int:
        return hm_color_boxes(self.ctx, level)

    def sample(self, op: hm_op, level: int):
        hm_sample(self.ctx, op, level)

    def compress(self, op: hm_op, tol: float = 0.0, rank: int = 0):
        """Algorithm 4.1 (tol and rank both 0: the settings' tol and rank)."""
        hm_compress(self.ctx, op, tol, rank)
        return hm_get_info(self.ctx)

    def apply(self, x, trans: int = 0):
        """x: (n,) or (n, nrhs) float64 CUDA tensor in original order."""
        t = self.torch
        vec = x.dim() == 1
        X = x.reshape(x.shape[0], -1).to(dtype=t.float64)
        Xc = X.t().contiguous()              # column-major n x nrhs
        Yc = t.empty_like(Xc)
        hm_apply(self.ctx, Xc.data_ptr(), Yc.data_ptr(), X.shape[1], trans)
        Y = Yc.t()
        return Y[:, 0] if vec else Y

    def apply_noalloc(self, x, trans: int = 0):
        """Like apply(), through hm_apply_noalloc (no device allocation in the library)."""
        t = self.torch
        vec = x.dim() == 1
        X = x.reshape(x.shape[0], -1).to(dtype=t.float64)
        Xc = X.t().contiguous()
        Yc = t.empty_like(Xc)
        hm_apply_noalloc(self.ctx, Xc.data_ptr(), Yc.data_ptr(), X.shape[1], trans)
        Y = Yc.t()
        return Y[:, 0] if vec else Y

    def relerr(self, op: hm_op, iters: int = 20) -> float:
        return hm_relerr(self.ctx, op, iters)

    def info(self) -> hm_info:
        return hm_get_info(self.ctx)

    def export(self, what: int, level: int = 0) -> bytes:
        return hm_export(self.ctx, what, level)

    def export_into(self, what: int, level: int, out):
        """hm_export into a contiguous host torch tensor (pinned memory makes the
        copy fast); returns out viewed as raw bytes of the exported size."""
        need = hm_export_size(self.ctx, what, level)
        nbytes = out.numel() * out.element_size()
        if not out.is_contiguous() or out.device.type != "cpu" or nbytes < need:
            raise ValueError(f"export_into: need a contiguous host tensor of at least {need} bytes")
        hm_export_into(self.ctx, what, level, out.data_ptr(), nbytes)
        return need


# ---------------------------------------------------------------------------
# serving (hm_server_*)
# ---------------------------------------------------------------------------

class Server:
    """Compression jobs admitted by device-memory footprint, compressed
    concurrently (one stream each) and kept resident for matvecs."""

    def __init__(self, slots: int = 4, hbm_budget: int = 0):
        import torch
        self.torch = torch
        cfg = hm_server_config(hbm_budget, slots)
        h = ctypes.c_void_p()
        st = _lib.hm_server_create(ctypes.byref(h), ctypes.byref(cfg))
        if st != HM_OK:
            raise HMError(st, "hm_server_create", "")
        self.h = h
        self._keep = {}

    def submit(self, points, settings: Settings, op: hm_op, leaf_size: int = 0, tol: float = 0.0,
               rank: int = 0) -> int:
        """points: host array-like (n x d float64, original order)."""
        import numpy as np
        pts = np.ascontiguousarray(np.asarray(points, dtype=np.float64))
        desc = hm_job_desc(settings.to_c(), op, pts.ctypes.data, pts.shape[0], leaf_size, tol, rank)
        jid = ctypes.c_int64(0)
        st = _lib.hm_server_submit(self.h, ctypes.byref(desc), ctypes.byref(jid))
        if st != HM_OK:
            raise HMError(st, "hm_server_submit", "")
        self._keep[jid.value] = op  # a dense matrix or callback must outlive the job
        return jid.value

    def wait(self, job: int, timeout: float = -1.0) -> hm_job_stats:
        stats = hm_job_stats()
        st = _lib.hm_server_wait(self.h, job, timeout, ctypes.byref(stats))
        if st != HM_OK:
            raise HMError(st, "hm_server_wait", f"job {job}")
        return stats

    def apply(self, job: int, x, trans: int = 0):
        """x: (n,) or (n, nrhs) float64 CUDA tensor in original order; synchronous."""
        t = self.torch
        vec = x.dim() == 1
        X = x.reshape(x.shape[0], -1).to(dtype=t.float64)
        Xc = X.t().contiguous()
        Yc = t.empty_like(Xc)
        t.cuda.current_stream().synchronize()  # X is complete before the job's stream reads it
        st = _lib.hm_server_apply(self.h, job, Xc.data_ptr(), Yc.data_ptr(), X.shape[1], trans)
        if st != HM_OK:
            raise HMError(st, "hm_server_apply", f"job {job}")
        Y = Yc.t()
        return Y[:, 0] if vec else Y

    def release(self, job: int):
        st = _lib.hm_server_release(self.h, job)
        if st != HM_OK:
            raise HMError(st, "hm_server_release", f"job {job}")
        self._keep.pop(job, None)

    def info(self) -> hm_server_info:
        out = hm_server_info()
        _check(None, _lib.hm_server_get_info(self.h, ctypes.byref(out)), "hm_server_get_info")
        return out

    def close(self):
        if self.h:
            _lib.hm_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
