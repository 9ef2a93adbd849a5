"""Thin ctypes binding of libdfacto (include/dfacto.h).

Each function here has the name of the C entry point it calls and only
marshals arguments: torch tensors (CPU or CUDA) are passed by ``data_ptr()``,
streams by their ``cuda_stream`` handle.  All compute happens in the CUDA
library; if ``libdfacto.so`` has not been built, loading raises -- there is no
fallback path.

Statuses other than OK raise :class:`DfactoError`, except the two informational
ones (``ESINGULAR`` from ALS, ``ELSFAIL`` from GD), which are returned.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence, Tuple

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdfacto.so")

OK, EINVAL, ERANGE, EDUP, ENOMEM, ECUDA, ESINGULAR, ELSFAIL, ETIMEOUT, EINTERNAL = range(10)
BACKTRACKING, EXACT = 0, 1  # dfacto_options.line_search
F32, BF16, F64 = 0, 1, 2
_DTYPE = {torch.float32: F32, torch.bfloat16: BF16, torch.float64: F64}


class DfactoError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s (status %d)" % (message, status))
        self.status = status


class dfacto_options(ctypes.Structure):
    _fields_ = [("rank", ctypes.c_int32), ("factor_dtype", ctypes.c_int32),
                ("lambda_reg", ctypes.c_double), ("seg_nnz", ctypes.c_int32),
                ("vec", ctypes.c_int32), ("walk", ctypes.c_int32),
                ("line_search", ctypes.c_int32), ("reserved", ctypes.c_int32 * 4)]


class dfacto_info(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int32 * 3), ("rank", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("nfib", ctypes.c_int64 * 3), ("device_bytes", ctypes.c_int64),
                ("norm_x2", ctypes.c_double), ("factor_dtype", ctypes.c_int32),
                ("seg_nnz", ctypes.c_int32 * 3), ("vec", ctypes.c_int32 * 3)]


class dfacto_csr_view(ctypes.Structure):
    _fields_ = [("dim_o", ctypes.c_int64), ("nfib", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("fiber_ptr", ctypes.c_void_p), ("fiber_idx", ctypes.c_void_p),
                ("nz_ptr", ctypes.c_void_p), ("nz_idx", ctypes.c_void_p),
                ("nz_val", ctypes.c_void_p)]


class dfacto_ratings_view(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int64), ("nnz", ctypes.c_int64), ("ptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class dfacto_batch_options(ctypes.Structure):
    _fields_ = [("use_graph", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 6)]


class dfacto_batch_class(ctypes.Structure):
    _fields_ = [("rank", ctypes.c_int32), ("factor_dtype", ctypes.c_int32),
                ("n_jobs", ctypes.c_int32), ("vec", ctypes.c_int32), ("lanes", ctypes.c_int32),
                ("seg_nnz", ctypes.c_int32), ("nnz", ctypes.c_int64), ("tuned_ms", ctypes.c_double)]


_lib = None

# Every symbol the header declares, with its ctypes signature.
_P, _I, _I64, _D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
SIGNATURES = {
    "dfacto_options_init": (None, [_P, ctypes.c_int32]),
    "dfacto_status_str": (ctypes.c_char_p, [_I]),
    "dfacto_build": (_I, [_P, _P, _I64, _P, _P, _P, _P]),
    "dfacto_destroy": (None, [_P]),
    "dfacto_last_error": (ctypes.c_char_p, [_P]),
    "dfacto_launch_count": (ctypes.c_int64, []),
    "dfacto_get_info": (_I, [_P, _P]),
    "dfacto_set_stream": (_I, [_P, _P]),
    "dfacto_sync": (_I, [_P]),
    "dfacto_set_factors": (_I, [_P, _I, _P, _I]),
    "dfacto_get_factors": (_I, [_P, _I, _P, _I]),
    "dfacto_get_lambda": (_I, [_P, _P]),
    "dfacto_set_lambda": (_I, [_P, _P]),
    "dfacto_mttkrp": (_I, [_P, _I, _P]),
    "dfacto_als_iter": (_I, [_P, _P]),
    "dfacto_gd_iter": (_I, [_P, _P, _P]),
    "dfacto_fit": (_I, [_P, _P]),
    "dfacto_get_csr": (_I, [_P, _I, _P]),
    "dfacto_mttkrp_noalloc": (_I, [_P, _P, _P, ctypes.c_int32, _P, _P]),
    "dfacto_joint_set_ratings": (_I, [_P, _P, _P, _I64, _D]),
    "dfacto_get_ratings_csr": (_I, [_P, _I, _P]),
    "dfacto_joint_als_iter": (_I, [_P, _P]),
    "dfacto_joint_gd_iter": (_I, [_P, _P, _P]),
    "dfacto_joint_objective": (_I, [_P, _P]),
    "dfacto_batch_options_init": (None, [_P]),
    "dfacto_batch_create": (_I, [_P, ctypes.c_int32, _P, _P, _P]),
    "dfacto_batch_destroy": (None, [_P]),
    "dfacto_batch_mttkrp": (_I, [_P, _I, _P]),
    "dfacto_batch_als_iter": (_I, [_P, _P]),
    "dfacto_batch_sync": (_I, [_P]),
    "dfacto_batch_num_classes": (ctypes.c_int32, [_P]),
    "dfacto_batch_get_class": (_I, [_P, ctypes.c_int32, _P]),
    "dfacto_batch_last_error": (ctypes.c_char_p, [_P]),
}


def load(path: str = LIB_PATH):
    """Load libdfacto.so (raises if it is missing: build it first)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError("libdfacto.so not found at %s; run __graft_entry__.build()" % path)
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name, None)
            if fn is None:
                raise ImportError("%s does not export %s" % (path, name))
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(st: int, h=None, allow=(), batch=None) -> int:
    if st == OK or st in allow:
        return st
    msg = load().dfacto_status_str(st).decode()
    if batch is not None:
        detail = load().dfacto_batch_last_error(batch)
        if detail:
            msg += ": " + detail.decode()
    if h is not None:
        detail = load().dfacto_last_error(h)
        if detail:
            msg += ": " + detail.decode()
    raise DfactoError(st, msg)


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
        return None
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def dfacto_options_init(rank: int, factor_dtype: int = F32, lambda_reg: float = 0.0,
                        seg_nnz: int = 0, vec: int = 0, walk: int = 0,
                        line_search: int = 0) -> dfacto_options:
    opt = dfacto_options()
    load().dfacto_options_init(ctypes.byref(opt), int(rank))
    opt.factor_dtype = factor_dtype
    opt.lambda_reg = float(lambda_reg)
    opt.seg_nnz = int(seg_nnz)
    opt.vec = int(vec)
    opt.walk = int(walk)
    opt.line_search = int(line_search)
    return opt


def dfacto_status_str(status: int) -> str:
    return load().dfacto_status_str(int(status)).decode()


def dfacto_build(idx: torch.Tensor, val: torch.Tensor, dims: Sequence[int],
                 opt: Optional[dfacto_options] = None, stream=None) -> int:
    """idx int32 [3, nnz] (contiguous), val float32 [nnz]; CPU or CUDA tensors."""
    assert idx.dtype == torch.int32 and val.dtype == torch.float32
    idx = idx.contiguous()
    val = val.contiguous()
    nnz = int(val.numel())
    assert idx.numel() == 3 * nnz
    d = (ctypes.c_int32 * 3)(*[int(x) for x in dims])
    out = ctypes.c_void_p()
    st = load().dfacto_build(idx.data_ptr() if nnz else None, val.data_ptr() if nnz else None,
                             nnz, d, ctypes.byref(opt) if opt is not None else None,
                             _stream_ptr(stream), ctypes.byref(out))
    _check(st)
    return out.value


def dfacto_destroy(h) -> None:
    load().dfacto_destroy(h)


def dfacto_last_error(h) -> str:
    return load().dfacto_last_error(h).decode()


def dfacto_launch_count() -> int:
    return int(load().dfacto_launch_count())


def dfacto_get_info(h) -> dfacto_info:
    info = dfacto_info()
    _check(load().dfacto_get_info(h, ctypes.byref(info)), h)
    return info


def dfacto_set_stream(h, stream) -> None:
    _check(load().dfacto_set_stream(h, _stream_ptr(stream)), h)


def dfacto_sync(h) -> None:
    _check(load().dfacto_sync(h), h)


def dfacto_set_factors(h, mode: int, F: torch.Tensor) -> None:
    F = F.contiguous()
    _check(load().dfacto_set_factors(h, int(mode), F.data_ptr(), _DTYPE[F.dtype]), h)


def dfacto_get_factors(h, mode: int, out: torch.Tensor) -> torch.Tensor:
    assert out.is_contiguous()
    _check(load().dfacto_get_factors(h, int(mode), out.data_ptr(), _DTYPE[out.dtype]), h)
    return out


def dfacto_get_lambda(h, R: int):
    buf = (ctypes.c_double * R)()
    _check(load().dfacto_get_lambda(h, buf), h)
    return list(buf)


def dfacto_set_lambda(h, lam: Sequence[float]) -> None:
    buf = (ctypes.c_double * len(lam))(*[float(x) for x in lam])
    _check(load().dfacto_set_lambda(h, buf), h)


def dfacto_mttkrp(h, mode: int, out: torch.Tensor) -> torch.Tensor:
    assert out.is_cuda and out.dtype == torch.float32 and out.is_contiguous()
    _check(load().dfacto_mttkrp(h, int(mode), out.data_ptr()), h)
    return out


def dfacto_als_iter(h, want_fit: bool = True) -> Tuple[int, Optional[float]]:
    fit = ctypes.c_double(0.0)
    st = load().dfacto_als_iter(h, ctypes.byref(fit) if want_fit else None)
    st = _check(st, h, allow=(ESINGULAR,))
    return st, (fit.value if want_fit else None)


def dfacto_gd_iter(h, want: bool = True) -> Tuple[int, Optional[float], Optional[float]]:
    loss = ctypes.c_double(0.0)
    alpha = ctypes.c_double(0.0)
    if want:
        st = load().dfacto_gd_iter(h, ctypes.byref(loss), ctypes.byref(alpha))
    else:
        st = load().dfacto_gd_iter(h, None, None)
    st = _check(st, h, allow=(ELSFAIL,))
    return st, (loss.value if want else None), (alpha.value if want else None)


def dfacto_fit(h) -> float:
    fit = ctypes.c_double(0.0)
    _check(load().dfacto_fit(h, ctypes.byref(fit)), h)
    return fit.value


def dfacto_get_csr(h, mode: int) -> dfacto_csr_view:
    v = dfacto_csr_view()
    _check(load().dfacto_get_csr(h, int(mode), ctypes.byref(v)), h)
    return v


def device_view(ptr: int, n: int, dtype: torch.dtype) -> torch.Tensor:
    """A torch view (no copy) of n elements of library-owned device memory."""
    typestr = {torch.int64: "<i8", torch.int32: "<i4", torch.float32: "<f4",
               torch.float64: "<f8"}[dtype]

    class _Iface:
        __cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr,
                                    "data": (int(ptr or 0), False), "version": 2}
    if n == 0:
        return torch.empty(0, dtype=dtype, device="cuda")
    return torch.as_tensor(_Iface(), device="cuda")


def dfacto_mttkrp_noalloc(csr: dfacto_csr_view, F_in: torch.Tensor, F_f: torch.Tensor, R: int,
                          out: torch.Tensor, stream=None) -> torch.Tensor:
    """MTTKRP of one mode without any device allocation (scratch in the
    library's fixed 16 MiB device array); arguments as in include/dfacto.h."""
    for t in (F_in, F_f, out):
        assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
    st = load().dfacto_mttkrp_noalloc(ctypes.byref(csr), F_in.data_ptr(), F_f.data_ptr(), int(R),
                                      out.data_ptr(), _stream_ptr(stream))
    if st == ENOMEM:
        raise DfactoError(st, "dfacto_mttkrp_noalloc: the problem needs more scratch than the "
                              "library's fixed 16 MiB device array holds")
    _check(st)
    return out


def dfacto_joint_set_ratings(h, yidx: torch.Tensor, yval: torch.Tensor, mu: float) -> None:
    """yidx int32 [2, nnzY] (user, item), yval float32 [nnzY]; CPU or CUDA tensors."""
    assert yidx.dtype == torch.int32 and yval.dtype == torch.float32
    yidx = yidx.contiguous()
    yval = yval.contiguous()
    n = int(yval.numel())
    assert yidx.numel() == 2 * n
    _check(load().dfacto_joint_set_ratings(h, yidx.data_ptr() if n else None,
                                           yval.data_ptr() if n else None, n, float(mu)), h)


def dfacto_get_ratings_csr(h, side: int) -> dfacto_ratings_view:
    v = dfacto_ratings_view()
    _check(load().dfacto_get_ratings_csr(h, int(side), ctypes.byref(v)), h)
    return v


def dfacto_joint_als_iter(h, want: bool = True) -> Optional[float]:
    obj = ctypes.c_double(0.0)
    _check(load().dfacto_joint_als_iter(h, ctypes.byref(obj) if want else None), h)
    return obj.value if want else None


def dfacto_joint_gd_iter(h, want: bool = True) -> Tuple[int, Optional[float], Optional[float]]:
    obj = ctypes.c_double(0.0)
    alpha = ctypes.c_double(0.0)
    if want:
        st = load().dfacto_joint_gd_iter(h, ctypes.byref(obj), ctypes.byref(alpha))
    else:
        st = load().dfacto_joint_gd_iter(h, None, None)
    st = _check(st, h, allow=(ELSFAIL,))
    return st, (obj.value if want else None), (alpha.value if want else None)


def dfacto_joint_objective(h) -> float:
    obj = ctypes.c_double(0.0)
    _check(load().dfacto_joint_objective(h, ctypes.byref(obj)), h)
    return obj.value


def ratings_to_tensors(view: dfacto_ratings_view) -> dict:
    """Copies (torch tensors on the GPU) of the arrays of a ratings CSR view."""
    torch.cuda.synchronize()
    return dict(ptr=device_view(view.ptr, view.rows + 1, torch.int64).clone(),
                col=device_view(view.col, view.nnz, torch.int32).clone(),
                val=device_view(view.val, view.nnz, torch.float32).clone())


def csr_to_tensors(view: dfacto_csr_view) -> dict:
    """Copies (torch tensors on the GPU) of the arrays of a CSR view."""
    torch.cuda.synchronize()
    return dict(fiber_ptr=device_view(view.fiber_ptr, view.dim_o + 1, torch.int64).clone(),
                fiber_idx=device_view(view.fiber_idx, view.nfib, torch.int32).clone(),
                nz_ptr=device_view(view.nz_ptr, view.nfib + 1, torch.int64).clone(),
                nz_idx=device_view(view.nz_idx, view.nnz, torch.int32).clone(),
                nz_val=device_view(view.nz_val, view.nnz, torch.float32).clone(),
                nfib=int(view.nfib))


class Tensor:
    """Owning wrapper of a dfacto handle (destroyed with the object)."""

    def __init__(self, idx, val, dims, rank: int, factor_dtype: int = F32,
                 lambda_reg: float = 0.0, seg_nnz: int = 0, vec: int = 0, walk: int = 0,
                 line_search: int = 0, stream=None):
        self.dims = [int(d) for d in dims]
        self.rank = int(rank)
        self.opt = dfacto_options_init(rank, factor_dtype, lambda_reg, seg_nnz, vec, walk,
                                       line_search)
        self.h = dfacto_build(idx, val, dims, self.opt, stream)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            dfacto_destroy(h)
            self.h = None

    def set_factors(self, factors) -> None:
        for m, F in enumerate(factors):
            dfacto_set_factors(self.h, m, F)

    # joint matrix completion + tensor factorization (Appendix F)
    def set_ratings(self, yidx, yval, mu: float) -> None:
        dfacto_joint_set_ratings(self.h, yidx, yval, mu)

    def joint_als_iter(self, want: bool = True):
        return dfacto_joint_als_iter(self.h, want)

    def joint_gd_iter(self, want: bool = True):
        return dfacto_joint_gd_iter(self.h, want)

    def joint_objective(self) -> float:
        return dfacto_joint_objective(self.h)

    def factors(self, dtype=torch.float32, device="cuda"):
        return [dfacto_get_factors(self.h, m, torch.empty(d, self.rank, dtype=dtype, device=device))
                for m, d in enumerate(self.dims)]

    def mttkrp(self, mode: int, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        if out is None:
            out = torch.empty(self.dims[mode], self.rank, dtype=torch.float32, device="cuda")
        return dfacto_mttkrp(self.h, mode, out)

    def als_iter(self, want_fit: bool = True):
        return dfacto_als_iter(self.h, want_fit)

    def gd_iter(self, want: bool = True):
        return dfacto_gd_iter(self.h, want)

    def fit(self) -> float:
        return dfacto_fit(self.h)

    def lam(self):
        return dfacto_get_lambda(self.h, self.rank)

    def info(self) -> dfacto_info:
        return dfacto_get_info(self.h)

    def csr(self, mode: int) -> dict:
        return csr_to_tensors(dfacto_get_csr(self.h, mode))


# ---- batches -----------------------------------------------------------------

def dfacto_batch_options_init(use_graph: bool = True, autotune: bool = True) -> dfacto_batch_options:
    opt = dfacto_batch_options()
    load().dfacto_batch_options_init(ctypes.byref(opt))
    opt.use_graph = int(bool(use_graph))
    opt.autotune = int(bool(autotune))
    return opt


def dfacto_batch_create(handles: Sequence, opt: Optional[dfacto_batch_options] = None, stream=None):
    arr = (ctypes.c_void_p * len(handles))(*[ctypes.c_void_p(h) for h in handles])
    out = ctypes.c_void_p()
    st = load().dfacto_batch_create(arr, len(handles), ctypes.byref(opt) if opt is not None else None,
                                    _stream_ptr(stream), ctypes.byref(out))
    _check(st)
    return out.value


def dfacto_batch_destroy(b) -> None:
    if b:
        load().dfacto_batch_destroy(b)


def dfacto_batch_mttkrp(b, mode: int, outs: Sequence[torch.Tensor]) -> Sequence[torch.Tensor]:
    for t in outs:
        assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
    arr = (ctypes.c_void_p * len(outs))(*[t.data_ptr() for t in outs])
    _check(load().dfacto_batch_mttkrp(b, int(mode), arr), batch=b)
    return outs


def dfacto_batch_als_iter(b, n: int, want_fits: bool = True) -> Tuple[int, Optional[List[float]]]:
    fits = (ctypes.c_double * n)() if want_fits else None
    st = _check(load().dfacto_batch_als_iter(b, fits), allow=(ESINGULAR,), batch=b)
    return st, (list(fits) if want_fits else None)


def dfacto_batch_sync(b) -> None:
    _check(load().dfacto_batch_sync(b), batch=b)


def dfacto_batch_classes(b) -> List[dfacto_batch_class]:
    out = []
    for k in range(load().dfacto_batch_num_classes(b)):
        c = dfacto_batch_class()
        _check(load().dfacto_batch_get_class(b, k, ctypes.byref(c)), batch=b)
        out.append(c)
    return out


class Batch:
    """Owning wrapper of a batch of Tensor jobs.  Holds references to the jobs
    so that they outlive the batch (the batch must be destroyed first)."""

    def __init__(self, tensors: Sequence["Tensor"], use_graph: bool = True, autotune: bool = True,
                 stream=None):
        self.tensors = list(tensors)
        self.opt = dfacto_batch_options_init(use_graph, autotune)
        self.b = dfacto_batch_create([t.h for t in self.tensors], self.opt, stream)

    def close(self) -> None:
        b = getattr(self, "b", None)
        if b:
            dfacto_batch_destroy(b)
            self.b = None

    def __del__(self):
        self.close()

    def mttkrp(self, mode: int, outs: Optional[Sequence[torch.Tensor]] = None):
        if outs is None:
            outs = [torch.empty(t.dims[mode], t.rank, dtype=torch.float32, device="cuda")
                    for t in self.tensors]
        return dfacto_batch_mttkrp(self.b, mode, outs)

    def als_iter(self, want_fits: bool = True):
        return dfacto_batch_als_iter(self.b, len(self.tensors), want_fits)

    def sync(self) -> None:
        dfacto_batch_sync(self.b)

    def classes(self) -> List[dfacto_batch_class]:
        return dfacto_batch_classes(self.b)
