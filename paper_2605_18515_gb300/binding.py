"""ctypes binding of the cbspmv C ABI (include/cbspmv.h).

Argument marshalling only: every step of the analysis and of the product runs inside
libcbspmv.so. PyTorch provides device memory and streams. If the library is missing the
import of this module raises; there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

CBSPMV_OK = 0
(CBSPMV_ERR_INVALID, CBSPMV_ERR_NOT_CANONICAL, CBSPMV_ERR_OOM, CBSPMV_ERR_CUDA, CBSPMV_ERR_TIMEOUT,
 CBSPMV_ERR_UNSUPPORTED, CBSPMV_ERR_BUSY) = range(1, 8)
STATUS = {0: "OK", 1: "ERR_INVALID", 2: "ERR_NOT_CANONICAL", 3: "ERR_OOM", 4: "ERR_CUDA",
          5: "ERR_TIMEOUT", 6: "ERR_UNSUPPORTED", 7: "ERR_BUSY"}
DTYPES = {"f64": 0, "f32": 1, "bf16": 2, "f16": 3}
FMT_NAMES = ("COO", "CSR", "DENSE")


class CbspmvError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Csr(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p), ("val", ctypes.c_void_p),
                ("on_device", ctypes.c_int)]


class Opts(ctypes.Structure):
    _fields_ = [("th0", ctypes.c_double), ("th1", ctypes.c_int), ("th2", ctypes.c_int),
                ("col_agg", ctypes.c_int), ("value_dtype", ctypes.c_int), ("unit_work", ctypes.c_int),
                ("load_balance", ctypes.c_int), ("device", ctypes.c_int), ("keep_value_map", ctypes.c_int),
                ("record_layout", ctypes.c_int), ("plain_records", ctypes.c_int), ("reserved", ctypes.c_int * 5)]


class Stats(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("n_block_rows", ctypes.c_int64), ("n_tiles", ctypes.c_int64),
                ("n_tiles_plain", ctypes.c_int64), ("super_sparse_fraction", ctypes.c_double),
                ("aggregated", ctypes.c_int), ("value_dtype", ctypes.c_int),
                ("n_fmt", ctypes.c_int64 * 3), ("nnz_fmt", ctypes.c_int64 * 3),
                ("hist_coarse", ctypes.c_int64 * 8), ("hist_fine", ctypes.c_int64 * 4),
                ("restore_cols_len", ctypes.c_int64), ("stream_bytes", ctypes.c_int64),
                ("metadata_bytes", ctypes.c_int64), ("model_bytes_cb", ctypes.c_int64),
                ("model_bytes_csr", ctypes.c_int64), ("model_bytes_bsr16", ctypes.c_int64),
                ("algo_bytes_per_run", ctypes.c_int64), ("flops_per_run", ctypes.c_int64),
                ("mults_per_run", ctypes.c_int64), ("n_units", ctypes.c_int64),
                ("n_split_units", ctypes.c_int64), ("n_split_rows", ctypes.c_int64),
                ("n_workers", ctypes.c_int64), ("worker_load_max", ctypes.c_double),
                ("worker_load_mean", ctypes.c_double), ("worker_load_std", ctypes.c_double),
                ("tb8_load_std", ctypes.c_double), ("analyze_ms", ctypes.c_double),
                ("n_entry_mode_units", ctypes.c_int64), ("n_xseq_units", ctypes.c_int64),
                ("fma_slots", ctypes.c_int64), ("n_direct_units", ctypes.c_int64),
                ("lane_layout", ctypes.c_int64), ("analyzed_on_device", ctypes.c_int64),
                ("n_g16_units", ctypes.c_int64), ("gather_list_bytes", ctypes.c_int64)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("memory_budget", ctypes.c_int64), ("max_inflight", ctypes.c_int),
                ("cg_inner_dtype", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("inner_max_iter", ctypes.c_int), ("max_outer", ctypes.c_int),
                ("inner_steps", ctypes.c_int), ("max_inflight_cg", ctypes.c_int), ("cg_oldest_first", ctypes.c_int),
                ("reserved", ctypes.c_int * 5)]


class Request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("matrix", ctypes.c_int), ("inp", ctypes.c_void_p),
                ("out", ctypes.c_void_p), ("alpha", ctypes.c_double), ("beta", ctypes.c_double),
                ("tol", ctypes.c_double), ("reserved", ctypes.c_int * 4)]


class Result(ctypes.Structure):
    _fields_ = [("done", ctypes.c_int), ("status", ctypes.c_int), ("iterations", ctypes.c_int),
                ("refinements", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("submitted", "admitted", "completed", "ticks", "launches",
                                              "max_inflight_seen", "arena_used_max", "arena_capacity",
                                              "queued", "inflight")]


REQ_SPMV, REQ_CG = 0, 1

class TuneReport(ctypes.Structure):
    _fields_ = [("n_tried", ctypes.c_int), ("default_ms", ctypes.c_double), ("best_ms", ctypes.c_double),
                ("best_unit_work", ctypes.c_int), ("best_col_agg", ctypes.c_int), ("best_th1", ctypes.c_int),
                ("best_th2", ctypes.c_int), ("tried_ms", ctypes.c_double * 16),
                ("tried_unit_work", ctypes.c_int * 16), ("tried_col_agg", ctypes.c_int * 16),
                ("tried_th1", ctypes.c_int * 16), ("tried_th2", ctypes.c_int * 16),
                ("best_record_layout", ctypes.c_int), ("tried_record_layout", ctypes.c_int * 16)]


# Every entry point the header declares, with its ctypes signature.
_P, _D, _I, _I64 = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_int64
SIGNATURES = {
    "cbspmv_default_opts": [ctypes.POINTER(Opts)],
    "cbspmv_analyze": [ctypes.POINTER(Csr), ctypes.POINTER(Opts), _P, ctypes.POINTER(_P)],
    "cbspmv_run": [_P, _P, _P, _D, _D, _P],
    "cbspmv_run_host": [_P, _P, _P, _D, _D, _P],
    "cbspmv_run_noalloc": [_P, _P, _P, _D, _D, _P],
    "cbspmv_run_multi": [_P, _I, _P, _I64, _P, _I64, _D, _D, _P],
    "cbspmv_time_kernels": [_P, _P, _P, _D, _D, _I, _P, _P, _P, _P],
    "cbspmv_graph_create": [_I, _P, _P, _P, _P, _P, _P, ctypes.POINTER(_P)],
    "cbspmv_graph_launch": [_P, _P],
    "cbspmv_graph_destroy": [_P],
    "cbspmv_analyze_tuned": [ctypes.POINTER(Csr), ctypes.POINTER(Opts), _P, _I, ctypes.POINTER(_P),
                             ctypes.POINTER(TuneReport)],
    "cbspmv_analyze_batched": [_I, _P, ctypes.POINTER(Opts), _P, _P],
    "cbspmv_run_batched": [_I, _P, _P, _P, _P, _P, _P, _P],
    "cbspmv_check_device": [_P, _P],
    "cbspmv_update_values": [_P, _P, _I, _P],
    "cbspmv_export_csr": [_P, _P, _P, _P],
    "cbspmv_export_blocked": [_P, _P, _P, _P, _P, _P, _P],
    "cbspmv_get_stats": [_P, ctypes.POINTER(Stats)],
    "cbspmv_destroy": [_P],
    "cbspmv_server_default_opts": [ctypes.POINTER(ServerOpts)],
    "cbspmv_server_create": [ctypes.POINTER(ServerOpts), ctypes.POINTER(_P)],
    "cbspmv_server_register": [_P, ctypes.POINTER(Csr), ctypes.POINTER(Opts), ctypes.POINTER(_I)],
    "cbspmv_server_submit": [_P, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)],
    "cbspmv_server_poll": [_P, ctypes.c_uint64, ctypes.POINTER(Result)],
    "cbspmv_server_wait": [_P, ctypes.c_uint64, _I, ctypes.POINTER(Result)],
    "cbspmv_server_get_stats": [_P, ctypes.POINTER(ServerStats)],
    "cbspmv_server_destroy": [_P],
    "cbspmv_measure_fp64_fma": [_I, _P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
    "cbspmv_spmm": [_P, _I, _P, _I64, _P, _I64, _D, _D, _P],
    "cbspmv_last_error": [],
    "cbspmv_version": [],
}


def load_library(path: str | None = None) -> ctypes.CDLL:
    path = path or _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libcbspmv.so not built ({path}); run paper_2605_18515_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, args in SIGNATURES.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_char_p if name in ("cbspmv_last_error", "cbspmv_version") else ctypes.c_int
    return lib


_lib: ctypes.CDLL | None = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


def _check(status: int):
    if status != CBSPMV_OK:
        raise CbspmvError(status, lib().cbspmv_last_error().decode())


def default_opts() -> Opts:
    o = Opts()
    _check(lib().cbspmv_default_opts(ctypes.byref(o)))
    return o


def _stream_ptr(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream or None
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


def _torch_dtype(vec: str):
    import torch
    return torch.float64 if vec == "f64" else torch.float32


def _dev_cols(t, k: int, rows: int, name: str, vec: str = "f64") -> tuple[int | None, int]:
    """(pointer, leading dimension) of a torch CUDA tensor of the vector type, shape
    (k, >= rows), whose rows are the k vectors (row stride = leading dimension, unit column
    stride)."""
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != _torch_dtype(vec) or not t.is_cuda:
        raise TypeError(f"{name} must be a {_torch_dtype(vec)} CUDA tensor")
    if t.dim() != 2 or t.shape[0] != k or t.shape[1] < rows or (t.shape[1] > 1 and t.stride(1) != 1):
        raise ValueError(f"{name} must have shape ({k}, >= {rows}) with unit column stride")
    ld = t.stride(0) if k > 1 else max(t.shape[1], rows)
    return (t.data_ptr() or None), int(ld)


def _csr_struct(A):
    """cbspmv_csr_t for A (numpy or host arrays, or CUDA torch tensors) plus the arrays
    that must stay alive while the struct is used."""
    try:
        import torch
        on_dev = isinstance(A.row_ptr, torch.Tensor) and A.row_ptr.is_cuda
    except ImportError:
        on_dev = False
    m, n = int(A.m), int(A.n)
    if on_dev:
        rp = A.row_ptr.contiguous().to(torch.int64)
        col = A.col.contiguous().to(torch.int32)
        val = A.val.contiguous().to(torch.float64)
        nnz = int(col.numel())
        csr = Csr(m, n, nnz, rp.data_ptr(), col.data_ptr() if nnz else None,
                  val.data_ptr() if nnz else None, 1)
    else:
        rp = np.ascontiguousarray(A.row_ptr, dtype=np.int64)
        col = np.ascontiguousarray(A.col, dtype=np.int32)
        val = np.ascontiguousarray(A.val, dtype=np.float64)
        nnz = int(rp[-1]) if rp.size else 0
        csr = Csr(m, n, nnz, rp.ctypes.data, col.ctypes.data, val.ctypes.data, 0)
    return csr, (rp, col, val), nnz


def _make_opts(th0=0.15, th1=32, th2=128, col_agg=-1, value_dtype="f64", unit_work=0,
               load_balance=True, device=0, keep_value_map=False, record_layout=False,
               plain_records=False) -> Opts:
    o = default_opts()
    o.th0, o.th1, o.th2, o.col_agg = th0, th1, th2, col_agg
    o.value_dtype = DTYPES[value_dtype]
    o.unit_work = unit_work
    o.load_balance = 1 if load_balance else 0
    o.device = device
    o.keep_value_map = 1 if keep_value_map else 0
    o.record_layout = int(record_layout)   # False/0 default, True/1 records, 2 lane streams
    o.plain_records = 1 if plain_records else 0
    return o


def _dev_ptr(t, n: int, name: str, vec: str = "f64") -> int | None:
    """Device pointer of a contiguous torch CUDA tensor holding >= n values of the vector
    type (float64 for FP64 handles, float32 for the reduced value types)."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor on the GPU")
    if t.dtype != _torch_dtype(vec) or not t.is_cuda or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {_torch_dtype(vec)} CUDA tensor")
    if t.numel() < n:
        raise ValueError(f"{name} has {t.numel()} elements, needs {n}")
    return t.data_ptr() or None


class BlockedMatrix:
    """An analysed matrix (cbspmv handle). `A` is any object with m, n, row_ptr, col, val
    (e.g. inputs.CSR). device=-1 gives a host-only handle (analysis and export only)."""

    def __init__(self, A, *, th0=0.15, th1=32, th2=128, col_agg=-1, value_dtype="f64",
                 unit_work=0, load_balance=True, device=0, stream=None, keep_value_map=False,
                 record_layout=False, plain_records=False):
        """A's arrays may be host arrays or CUDA torch tensors (device-resident input)."""
        self._h = ctypes.c_void_p(None)
        self.m, self.n = int(A.m), int(A.n)
        csr, _keep, self.nnz = _csr_struct(A)
        o = _make_opts(th0, th1, th2, col_agg, value_dtype, unit_work, load_balance, device, keep_value_map,
                       record_layout, plain_records)
        self.device = device
        self.value_dtype = value_dtype
        self.vec = "f64" if value_dtype == "f64" else "f32"
        s = _stream_ptr(stream) if (device >= 0 or csr.on_device) else None
        _check(lib().cbspmv_analyze(ctypes.byref(csr), ctypes.byref(o), s, ctypes.byref(self._h)))

    @classmethod
    def _adopt(cls, handle: int, m: int, n: int, nnz: int, device: int,
               value_dtype: str = "f64") -> "BlockedMatrix":
        self = cls.__new__(cls)
        self._h = ctypes.c_void_p(handle)
        self.m, self.n, self.nnz, self.device = m, n, nnz, device
        self.value_dtype = value_dtype
        self.vec = "f64" if value_dtype == "f64" else "f32"
        return self

    @property
    def vector_dtype(self):
        """numpy dtype of x and y: float64 for FP64 values, float32 for the reduced types."""
        return np.float64 if self.vec == "f64" else np.float32

    @property
    def handle(self) -> int:
        return self._h.value

    def run(self, x, y, alpha: float = 1.0, beta: float = 0.0, stream=None):
        """y <- alpha*A*x + beta*y on the device (asynchronous on the stream)."""
        _check(lib().cbspmv_run(self._h, _dev_ptr(x, self.n, "x", self.vec), _dev_ptr(y, self.m, "y", self.vec),
                                float(alpha), float(beta), _stream_ptr(stream)))
        return y

    def run_multi(self, X, Y, alpha: float = 1.0, beta: float = 0.0, stream=None):
        """Y <- alpha*A*X + beta*Y for k vectors: X of shape (k, n), Y of shape (k, m),
        float64 CUDA tensors whose rows are the vectors (row stride = leading dimension)."""
        k = int(X.shape[0])
        px, ldx = _dev_cols(X, k, self.n, "X", self.vec)
        py, ldy = _dev_cols(Y, k, self.m, "Y", self.vec)
        _check(lib().cbspmv_run_multi(self._h, k, px, ldx, py, ldy, float(alpha), float(beta),
                                      _stream_ptr(stream)))
        return Y

    def spmm(self, X, Y, alpha: float = 1.0, beta: float = 0.0, stream=None):
        """Y <- alpha*A*X + beta*Y on the tensor cores (BF16 handles analysed with
        plain_records): X of shape (n, k), Y of shape (m, k), row-major float32 CUDA tensors
        (row stride = leading dimension, unit column stride)."""
        if X.dim() != 2 or Y.dim() != 2 or X.shape[1] != Y.shape[1] or X.shape[0] < self.n or Y.shape[0] < self.m:
            raise ValueError("X must be (n, k) and Y (m, k)")
        if X.stride(1) != 1 or Y.stride(1) != 1 or X.dtype != Y.dtype:
            raise ValueError("X and Y must have unit column stride and one dtype")
        k = int(X.shape[1])
        _check(lib().cbspmv_spmm(self._h, k, X.data_ptr(), int(X.stride(0)), Y.data_ptr(), int(Y.stride(0)),
                                 float(alpha), float(beta), _stream_ptr(stream)))
        return Y

    def time_kernels(self, x, y, reps: int, alpha: float = 1.0, beta: float = 0.0, stream=None) -> dict:
        """Mean device time per run of each kernel of the product (CUDA events around every
        launch, on the run's stream)."""
        a, b, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
        _check(lib().cbspmv_time_kernels(self._h, _dev_ptr(x, self.n, "x", self.vec),
                                         _dev_ptr(y, self.m, "y", self.vec),
                                         float(alpha), float(beta), int(reps), _stream_ptr(stream),
                                         ctypes.byref(a), ctypes.byref(b), ctypes.byref(n)))
        return {"ms_main": a.value, "ms_combine": b.value, "launches_per_run": n.value}

    def run_host(self, x: np.ndarray, y: np.ndarray | None = None, alpha: float = 1.0,
                 beta: float = 0.0, stream=None) -> np.ndarray:
        """The product from host arrays of the vector type (copies in and out, synchronous)."""
        vt = self.vector_dtype
        x = np.ascontiguousarray(x, dtype=vt)
        if y is None:
            y = np.zeros(self.m, dtype=vt)
        if y.dtype != vt or not y.flags.c_contiguous:
            raise TypeError(f"y must be a contiguous {np.dtype(vt).name} array")
        _check(lib().cbspmv_run_host(self._h, x.ctypes.data, y.ctypes.data, float(alpha), float(beta),
                                     _stream_ptr(stream)))
        return y

    def update_values(self, val, stream=None):
        """New values (CSR order of the analysed matrix, FP64): a numpy array (copied in) or a
        float64 CUDA tensor, re-packed on the device (requires keep_value_map=True)."""
        try:
            import torch
            dev = isinstance(val, torch.Tensor) and val.is_cuda
        except ImportError:
            dev = False
        if dev:
            if val.dtype != torch.float64 or not val.is_contiguous() or val.numel() < self.nnz:
                raise TypeError("val must be a contiguous float64 CUDA tensor with nnz entries")
            ptr = val.data_ptr() or None
        else:
            val = np.ascontiguousarray(val, dtype=np.float64)
            if val.size < self.nnz:
                raise ValueError("val must hold nnz entries")
            self._val_keep = val
            ptr = val.ctypes.data
        s = _stream_ptr(stream) if self.device >= 0 else None
        _check(lib().cbspmv_update_values(self._h, ptr, 1 if dev else 0, s))

    def check_device(self, stream=None):
        _check(lib().cbspmv_check_device(self._h, _stream_ptr(stream)))

    def export_csr(self):
        rp = np.empty(self.m + 1, dtype=np.int64)
        col = np.empty(max(self.nnz, 1), dtype=np.int32)
        val = np.empty(max(self.nnz, 1), dtype=np.float64)
        _check(lib().cbspmv_export_csr(self._h, rp.ctypes.data, col.ctypes.data, val.ctypes.data))
        return rp, col[:self.nnz], val[:self.nnz]

    def stats(self) -> dict:
        s = Stats()
        _check(lib().cbspmv_get_stats(self._h, ctypes.byref(s)))
        out = {}
        for name, _ in Stats._fields_:
            v = getattr(s, name)
            out[name] = list(v) if hasattr(v, "__len__") else v
        return out

    def export_blocked(self) -> dict:
        st = self.stats()
        nt, nbr, rl = st["n_tiles"], st["n_block_rows"], st["restore_cols_len"]
        br = np.empty(nt, np.int32); bc = np.empty(nt, np.int32)
        nz = np.empty(nt, np.int32); ty = np.empty(nt, np.uint8)
        co = np.zeros(nbr + 1 if st["aggregated"] else 0, np.int64)
        rc = np.zeros(rl, np.int32)
        _check(lib().cbspmv_export_blocked(self._h, br.ctypes.data, bc.ctypes.data, nz.ctypes.data,
                                           ty.ctypes.data, co.ctypes.data if co.size else None,
                                           rc.ctypes.data if rc.size else None))
        return {"blk_row": br, "blk_col": bc, "nnz": nz, "type": ty, "cols_offset": co,
                "restore_cols": rc, "aggregated": bool(st["aggregated"])}

    def close(self):
        if self._h and self._h.value:
            _check(lib().cbspmv_destroy(self._h))
            self._h = ctypes.c_void_p(None)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def analyze_batched(mats, *, stream=None, **opts) -> list["BlockedMatrix"]:
    """cbspmv_analyze_batched over a list of CSR matrices with one set of options."""
    count = len(mats)
    structs = [_csr_struct(A) for A in mats]
    arr = (Csr * max(count, 1))(*[c for c, _, _ in structs])
    o = _make_opts(**opts)
    out = (ctypes.c_void_p * max(count, 1))()
    s = _stream_ptr(stream) if o.device >= 0 else None
    _check(lib().cbspmv_analyze_batched(count, ctypes.addressof(arr), ctypes.byref(o), s,
                                        ctypes.addressof(out)))
    vd = opts.get("value_dtype", "f64")
    return [BlockedMatrix._adopt(out[i], int(A.m), int(A.n), structs[i][2], o.device, vd)
            for i, A in enumerate(mats)]


def run_batched(mats, Xs, Ys, alphas, betas, *, stream=None):
    """cbspmv_run_batched: problem i computes Ys[i] <- alphas[i]*A_i*Xs[i] + betas[i]*Ys[i].
    Xs[i], Ys[i] are CUDA tensors of the matrix's vector type, 1-D (one vector) or
    (k_i, n_i) / (k_i, m_i) contiguous (k_i vectors)."""
    count, arrs = _batch_arrays(mats, Xs, Ys, alphas, betas)
    _check(lib().cbspmv_run_batched(count, *[ctypes.addressof(a) for a in arrs], _stream_ptr(stream)))


class Server:
    """A serving engine (cbspmv_server_*): resident matrices, requests from host arrays,
    continuous batching of in-flight requests on the device."""

    def __init__(self, device=0, memory_budget=4 << 30, max_inflight=64, cg_inner_dtype="bf16",
                 inner_tol=1e-4, inner_max_iter=2000, max_outer=30, inner_steps=8, max_inflight_cg=0,
                 cg_oldest_first=False):
        o = ServerOpts()
        _check(lib().cbspmv_server_default_opts(ctypes.byref(o)))
        o.device, o.memory_budget, o.max_inflight = device, int(memory_budget), max_inflight
        o.cg_inner_dtype = DTYPES[cg_inner_dtype]
        o.inner_tol, o.inner_max_iter, o.max_outer = inner_tol, inner_max_iter, max_outer
        o.inner_steps = inner_steps
        o.max_inflight_cg = max_inflight_cg
        o.cg_oldest_first = 1 if cg_oldest_first else 0
        self._s = ctypes.c_void_p(None)
        _check(lib().cbspmv_server_create(ctypes.byref(o), ctypes.byref(self._s)))
        self._keep: dict[int, tuple] = {}
        self.shapes: list[tuple[int, int]] = []

    def register(self, A, **opts) -> int:
        csr, _keep, _ = _csr_struct(A)
        o = _make_opts(**opts)
        mid = ctypes.c_int()
        _check(lib().cbspmv_server_register(self._s, ctypes.byref(csr), ctypes.byref(o), ctypes.byref(mid)))
        self.shapes.append((int(A.m), int(A.n)))
        return mid.value

    def _shape(self, mid: int) -> tuple[int, int]:
        # an unknown id is passed on for the library to reject
        return self.shapes[mid] if 0 <= mid < len(self.shapes) else (1, 1)

    def _submit(self, kind, mid, inp, out, alpha=1.0, beta=0.0, tol=0.0) -> int:
        q = Request(kind, mid, inp.ctypes.data, out.ctypes.data, float(alpha), float(beta), float(tol))
        t = ctypes.c_uint64()
        _check(lib().cbspmv_server_submit(self._s, ctypes.byref(q), ctypes.byref(t)))
        self._keep[t.value] = (inp, out)
        return t.value

    def submit_spmv(self, mid: int, x: np.ndarray, y: np.ndarray | None = None, alpha=1.0, beta=0.0):
        """y <- alpha A x + beta y; returns (ticket, y)."""
        m, n = self._shape(mid)
        x = np.ascontiguousarray(x, dtype=np.float64)
        if y is None:
            y = np.zeros(m, np.float64)
        return self._submit(REQ_SPMV, mid, x, y, alpha, beta), y

    def submit_cg(self, mid: int, b: np.ndarray, tol=1e-8):
        """Solves A x = b to ||b - A x|| <= tol ||b||; returns (ticket, x)."""
        m, n = self._shape(mid)
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros(n, np.float64)
        return self._submit(REQ_CG, mid, b, x, tol=tol), x

    def wait(self, ticket: int, timeout_ms: int = 60000) -> dict:
        r = Result()
        st = lib().cbspmv_server_wait(self._s, ticket, int(timeout_ms), ctypes.byref(r))
        if st == CBSPMV_OK:
            self._keep.pop(ticket, None)
        elif st != CBSPMV_ERR_TIMEOUT:
            _check(st)
        return {f: getattr(r, f) for f, _ in Result._fields_} | {"wait_status": st}

    def poll(self, ticket: int) -> dict:
        r = Result()
        _check(lib().cbspmv_server_poll(self._s, ticket, ctypes.byref(r)))
        if r.done:
            self._keep.pop(ticket, None)
        return {f: getattr(r, f) for f, _ in Result._fields_}

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().cbspmv_server_get_stats(self._s, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def close(self):
        if self._s and self._s.value:
            _check(lib().cbspmv_server_destroy(self._s))
            self._s = ctypes.c_void_p(None)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _batch_arrays(mats, Xs, Ys, alphas, betas):
    count = len(mats)
    n1 = max(count, 1)
    hs = (ctypes.c_void_p * n1)(*[M.handle for M in mats])
    ks = (ctypes.c_int * n1)()
    xp = (ctypes.c_void_p * n1)()
    yp = (ctypes.c_void_p * n1)()
    al = (ctypes.c_double * n1)(*[float(a) for a in alphas])
    be = (ctypes.c_double * n1)(*[float(b) for b in betas])
    for i, M in enumerate(mats):
        X, Y = Xs[i], Ys[i]
        k = 1 if X.dim() == 1 else int(X.shape[0])
        ks[i] = k
        xp[i] = _dev_ptr(X, k * M.n, f"X[{i}]", M.vec)
        yp[i] = _dev_ptr(Y, k * M.m, f"Y[{i}]", M.vec)
    return count, (hs, ks, xp, yp, al, be)


class Graph:
    """cbspmv_graph_*: the products of run_batched(mats, Xs, Ys, alphas, betas) captured into
    a CUDA graph; launch() replays them (current X contents, Y overwritten)."""

    def __init__(self, mats, Xs, Ys, alphas, betas):
        count, arrs = _batch_arrays(mats, Xs, Ys, alphas, betas)
        self._keep = (mats, Xs, Ys, arrs)
        self._g = ctypes.c_void_p(None)
        _check(lib().cbspmv_graph_create(count, *[ctypes.addressof(a) for a in arrs], ctypes.byref(self._g)))

    def launch(self, stream=None):
        _check(lib().cbspmv_graph_launch(self._g, _stream_ptr(stream)))

    def close(self):
        if self._g and self._g.value:
            _check(lib().cbspmv_graph_destroy(self._g))
            self._g = ctypes.c_void_p(None)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def analyze_tuned(A, *, reps=20, stream=None, **opts):
    """cbspmv_analyze_tuned: the fastest of a few analysis options; returns
    (BlockedMatrix, report dict)."""
    csr, _keep, nnz = _csr_struct(A)
    o = _make_opts(**opts)
    h = ctypes.c_void_p(None)
    rep = TuneReport()
    _check(lib().cbspmv_analyze_tuned(ctypes.byref(csr), ctypes.byref(o), _stream_ptr(stream), int(reps),
                                      ctypes.byref(h), ctypes.byref(rep)))
    n = min(rep.n_tried, 16)
    report = {"n_tried": rep.n_tried, "default_ms": rep.default_ms, "best_ms": rep.best_ms,
              "best": {"unit_work": rep.best_unit_work, "col_agg": rep.best_col_agg, "th1": rep.best_th1,
                       "th2": rep.best_th2, "record_layout": rep.best_record_layout},
              "tried": [{"ms": rep.tried_ms[i], "unit_work": rep.tried_unit_work[i],
                         "col_agg": rep.tried_col_agg[i], "th1": rep.tried_th1[i], "th2": rep.tried_th2[i],
                         "record_layout": rep.tried_record_layout[i]}
                        for i in range(n)]}
    M = BlockedMatrix._adopt(h.value, int(A.m), int(A.n), nnz, o.device, opts.get("value_dtype", "f64"))
    return M, report


def measure_fp64_fma(device: int = 0, stream=None) -> dict:
    """FP64 FMA rate of the device (GFLOP/s) and SM cycles per warp-wide FP64 FMA."""
    g, c = ctypes.c_double(), ctypes.c_double()
    _check(lib().cbspmv_measure_fp64_fma(device, _stream_ptr(stream), ctypes.byref(g), ctypes.byref(c)))
    return {"gflops": g.value, "cycles_per_warp_fma": c.value}


def version() -> str:
    return lib().cbspmv_version().decode()
