"""FP64 CPU oracle for DFacTo -- test infrastructure only.

This package wraps ``dfacto_oracle.c`` (a plain, slow, FP64 restatement of the
paper's MTTKRP, CSR construction, ALS, GD and fit) with ctypes + numpy.  Only the
tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import
it.  The CUDA library never imports, links or calls anything in here, and nothing
here imports the library: the two share no code.

Every array crossing into C is converted to a C-contiguous numpy array of the
stated dtype; factor matrices are float64, row-major (rows x R).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
from typing import Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dfacto_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OK, EINVAL, ERANGE, EDUP, ENOMEM, ESINGULAR, ELSFAIL = 0, 1, 2, 3, 4, 6, 7


_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle with gcc into oracle/liboracle.so (if stale).  With
    openmp=True, the same source with -fopenmp into oracle/liboracle_omp.so:
    the multi-core CPU timing baseline (its pragmas parallelise the per-nonzero
    sums with per-thread partial sums, so only the summation order differs;
    the tests use the single-threaded build)."""
    lib = _LIB_OMP if openmp else _LIB
    if (not force and os.path.exists(lib)
            and os.path.getmtime(lib) >= os.path.getmtime(_SRC)):
        return lib
    tmp = lib + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    if openmp:
        cmd.insert(1, "-fopenmp")
    subprocess.check_call(cmd)
    os.replace(tmp, lib)
    return lib


_lib = None


def _load():
    global _lib
    if _lib is None:
        # DFACTO_ORACLE_LIB points the wrapper at another build of the same source
        # (the mutation tests load deliberately broken copies this way).
        path = os.environ.get("DFACTO_ORACLE_LIB")
        if not path:
            path = build()
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        I32 = ctypes.c_int
        D = ctypes.c_double
        sig = {
            "orc_check_coo": (I32, [I64, P, P]),
            "orc_build_csr": (I32, [I32, I64, P, P, P, P, P, P, P, P, P]),
            "orc_mttkrp": (None, [I32, I64, P, P, P, I32, P, P, P, P]),
            "orc_mttkrp_rows": (I32, [I32, I64, P, P, P, I32, P, P, P, I64, P, P]),
            "orc_gram": (None, [I64, I32, P, P]),
            "orc_sym_eig_jacobi": (I32, [I32, P, P, P]),
            "orc_pinv_sym": (I32, [I32, P, P]),
            "orc_solve_normal": (I32, [I64, I32, P, P, P]),
            "orc_als_mode_update": (I32, [I32, I64, P, P, P, I32, D, P, P, P, P]),
            "orc_als_sweep": (I32, [I64, P, P, P, I32, D, P, P, P, P, P]),
            "orc_norm2": (D, [I64, P]),
            "orc_inner": (D, [I64, P, P, I32, P, P, P, P]),
            "orc_model_norm2": (D, [P, I32, P, P, P, P]),
            "orc_fit": (D, [I64, P, P, P, I32, P, P, P, P]),
            "orc_loss": (D, [I64, P, P, P, I32, D, P, P, P]),
            "orc_gd_gradient": (I32, [I64, P, P, P, I32, D, P, P, P, P, P, P]),
            "orc_gd_step": (I32, [I64, P, P, P, I32, D, P, P, P, P, P, P]),
            "orc_gd_ray_poly": (I32, [I64, P, P, P, I32, D, P, P, P, P, P, P, P]),
            "orc_joint_loss": (D, [I64, P, P, I64, P, P, P, I32, D, D, P, P, P]),
            "orc_joint_gradient": (I32, [I64, P, P, I64, P, P, P, I32, D, D, P, P, P, P, P, P]),
            "orc_joint_als_sweep": (I32, [I64, P, P, I64, P, P, P, I32, D, D, P, P, P]),
            "orc_joint_gd_step": (I32, [I64, P, P, I64, P, P, P, I32, D, D, P, P, P, P, P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class Tensor:
    """A COO tensor as the oracle sees it: idx int32[3, nnz], val float32[nnz]."""

    def __init__(self, idx, val, dims: Sequence[int]):
        self.idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int32).reshape(3, -1))
        self.val = np.ascontiguousarray(np.asarray(val, dtype=np.float32).reshape(-1))
        self.dims = np.ascontiguousarray(np.asarray(dims, dtype=np.int32).reshape(3))
        self.nnz = int(self.val.shape[0])
        assert self.idx.shape[1] == self.nnz


def _f64(a, rows: int, R: int) -> np.ndarray:
    out = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    assert out.shape == (rows, R), (out.shape, rows, R)
    return out


def axes(mode: int) -> Tuple[int, int, int]:
    """(o, in, f) axes of mode n: o = n, in = n+1, f = n+2 (mod 3)."""
    return mode, (mode + 1) % 3, (mode + 2) % 3


def check_coo(t: Tensor) -> int:
    return _load().orc_check_coo(t.nnz, _p(t.idx), _p(t.dims))


def build_csr(t: Tensor, mode: int):
    """Return (status, dict of CSR arrays) for mode 0, 1 or 2."""
    lib = _load()
    o = mode
    n = max(t.nnz, 1)
    fiber_ptr = np.zeros(int(t.dims[o]) + 1, np.int64)
    fiber_idx = np.zeros(n, np.int32)
    nz_ptr = np.zeros(n + 1, np.int64)
    nz_idx = np.zeros(n, np.int32)
    nz_val = np.zeros(n, np.float32)
    nfib = np.zeros(1, np.int64)
    st = lib.orc_build_csr(mode, t.nnz, _p(t.idx), _p(t.val), _p(t.dims), _p(fiber_ptr),
                           _p(fiber_idx), _p(nz_ptr), _p(nz_idx), _p(nz_val), _p(nfib))
    if st != OK:
        return st, None
    nf = int(nfib[0])
    return st, dict(fiber_ptr=fiber_ptr, fiber_idx=fiber_idx[:nf].copy(),
                    nz_ptr=nz_ptr[:nf + 1].copy(), nz_idx=nz_idx[:t.nnz].copy(),
                    nz_val=nz_val[:t.nnz].copy(), nfib=nf)


def mttkrp(t: Tensor, mode: int, factors: Sequence[np.ndarray]) -> np.ndarray:
    R = int(np.asarray(factors[0]).shape[1])
    F = [_f64(factors[m], int(t.dims[m]), R) for m in range(3)]
    out = np.zeros((int(t.dims[mode]), R), np.float64)
    _load().orc_mttkrp(mode, t.nnz, _p(t.idx), _p(t.val), _p(t.dims), R,
                       _p(F[0]), _p(F[1]), _p(F[2]), _p(out))
    return out


def mttkrp_rows(t: Tensor, mode: int, factors: Sequence[np.ndarray], rows) -> np.ndarray:
    R = int(np.asarray(factors[0]).shape[1])
    F = [_f64(factors[m], int(t.dims[m]), R) for m in range(3)]
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    out = np.zeros((rows.shape[0], R), np.float64)
    st = _load().orc_mttkrp_rows(mode, t.nnz, _p(t.idx), _p(t.val), _p(t.dims), R,
                                 _p(F[0]), _p(F[1]), _p(F[2]), rows.shape[0], _p(rows),
                                 _p(out))
    if st != OK:
        raise ValueError("orc_mttkrp_rows status %d" % st)
    return out


def gram(F: np.ndarray) -> np.ndarray:
    F = np.ascontiguousarray(np.asarray(F, dtype=np.float64))
    R = F.shape[1]
    G = np.zeros((R, R), np.float64)
    _load().orc_gram(F.shape[0], R, _p(F), _p(G))
    return G


def sym_eig_jacobi(S: np.ndarray):
    A = np.ascontiguousarray(np.array(S, dtype=np.float64))
    R = A.shape[0]
    V = np.zeros((R, R), np.float64)
    w = np.zeros(R, np.float64)
    _load().orc_sym_eig_jacobi(R, _p(A), _p(V), _p(w))
    return w, V


def pinv_sym(S: np.ndarray) -> np.ndarray:
    S = np.ascontiguousarray(np.asarray(S, dtype=np.float64))
    P = np.zeros_like(S)
    _load().orc_pinv_sym(S.shape[0], _p(S), _p(P))
    return P


def solve_normal(Gamma: np.ndarray, N: np.ndarray):
    Gamma = np.ascontiguousarray(np.asarray(Gamma, dtype=np.float64))
    N = np.ascontiguousarray(np.asarray(N, dtype=np.float64))
    X = np.zeros_like(N)
    st = _load().orc_solve_normal(N.shape[0], N.shape[1], _p(Gamma), _p(N), _p(X))
    return st, X


def _factors_rw(t: Tensor, factors):
    R = int(np.asarray(factors[0]).shape[1])
    return R, [np.array(_f64(factors[m], int(t.dims[m]), R)) for m in range(3)]


def als_mode_update(t: Tensor, mode: int, factors, lambda_reg: float = 0.0):
    """Returns (status, [A,B,C] updated copies, lambda)."""
    R, F = _factors_rw(t, factors)
    lam = np.zeros(R, np.float64)
    st = _load().orc_als_mode_update(mode, t.nnz, _p(t.idx), _p(t.val), _p(t.dims), R,
                                     float(lambda_reg), _p(F[0]), _p(F[1]), _p(F[2]),
                                     _p(lam))
    return st, F, lam


def als_sweep(t: Tensor, factors, lambda_reg: float = 0.0):
    """Returns (status, [A,B,C] updated copies, lambda, fit)."""
    R, F = _factors_rw(t, factors)
    lam = np.zeros(R, np.float64)
    fit = np.zeros(1, np.float64)
    st = _load().orc_als_sweep(t.nnz, _p(t.idx), _p(t.val), _p(t.dims), R,
                               float(lambda_reg), _p(F[0]), _p(F[1]), _p(F[2]), _p(lam),
                               _p(fit))
    return st, F, lam, float(fit[0])


def norm2(t: Tensor) -> float:
    return _load().orc_norm2(t.nnz, _p(t.val))


def inner(t: Tensor, factors, lam=None) -> float:
    R = int(np.asarray(factors[0]).shape[1])
    F = [_f64(factors[m], int(t.dims[m]), R) for m in range(3)]
    lam = None if lam is None else np.ascontiguousarray(np.asarray(lam, np.float64))
    return _load().orc_inner(t.nnz, _p(t.idx), _p(t.val), R, _p(lam), _p(F[0]), _p(F[1]),
                             _p(F[2]))


def model_norm2(dims, factors, lam=None) -> float:
    R = int(np.asarray(factors[0]).shape[1])
    dims = np.ascontiguousarray(np.asarray(dims, np.int32))
    F = [_f64(factors[m], int(dims[m]), R) for m in range(3)]
    lam = None if lam is None else np.ascontiguousarray(np.asarray(lam, np.float64))
    return _load().orc_model_norm2(_p(dims), R, _p(lam), _p(F[0]), _p(F[1]), _p(F[2]))


def fit(t: Tensor, factors, lam=None) -> float:
    R = int(np.asarray(factors[0]).shape[1])
    F = [_f64(factors[m], int(t.dims[m]), R) for m in range(3)]
    lam = None if lam is None else np.ascontiguousarray(np.asarray(lam, np.float64))
    return _load().orc_fit(t.nnz, _p(t.idx), _p(t.val), _p(t.dims), R, _p(lam), _p(F[0]),
                           _p(F[1]), _p(F[2]))


def loss(t: Tensor, factors, lambda_reg: float = 0.0) -> float:
    R = int(np.asarray(factors[0]).shape[1])
    F = [_f64(factors[m], int(t.dims[m]), R) for m in range(3)]
    return _load().orc_loss(t.nnz, _p(t.idx), _p(t.val), _p(t.dims), R, float(lambda_reg),
                            _p(F[0]), _p(F[1]), _p(F[2]))


def gd_gradient(t: Tensor, factors, lambda_reg: float = 0.0):
    R = int(np.asarray(factors[0]).shape[1])
    F = [_f64(factors[m], int(t.dims[m]), R) for m in range(3)]
    G = [np.zeros_like(F[m]) for m in range(3)]
    st = _load().orc_gd_gradient(t.nnz, _p(t.idx), _p(t.val), _p(t.dims), R,
                                 float(lambda_reg), _p(F[0]), _p(F[1]), _p(F[2]), _p(G[0]),
                                 _p(G[1]), _p(G[2]))
    if st != OK:
        raise MemoryError("orc_gd_gradient status %d" % st)
    return G


def gd_step(t: Tensor, factors, alpha_prev: float = 0.0, lambda_reg: float = 0.0):
    """Returns (status, [A,B,C] updated copies, alpha, loss, g2)."""
    R, F = _factors_rw(t, factors)
    a = np.array([alpha_prev], np.float64)
    lo = np.zeros(1, np.float64)
    g2 = np.zeros(1, np.float64)
    st = _load().orc_gd_step(t.nnz, _p(t.idx), _p(t.val), _p(t.dims), R, float(lambda_reg),
                             _p(F[0]), _p(F[1]), _p(F[2]), _p(a), _p(lo), _p(g2))
    return st, F, float(a[0]), float(lo[0]), float(g2[0])


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))


def gd_ray_poly(t: Tensor, factors, grads, lambda_reg: float = 0.0) -> np.ndarray:
    """Coefficients c[0..6] of phi(alpha) = f(theta - alpha grad), lowest first
    (orc_gd_ray_poly: the objective's terms expanded in alpha)."""
    R = int(np.asarray(factors[0]).shape[1])
    F = [_f64(factors[m], int(t.dims[m]), R) for m in range(3)]
    G = [_f64(grads[m], int(t.dims[m]), R) for m in range(3)]
    c = np.zeros(7, np.float64)
    st = _load().orc_gd_ray_poly(t.nnz, _p(t.idx), _p(t.val), _p(t.dims), R, float(lambda_reg),
                                 _p(F[0]), _p(F[1]), _p(F[2]), _p(G[0]), _p(G[1]), _p(G[2]),
                                 _p(c))
    if st != OK:
        raise MemoryError("orc_gd_ray_poly status %d" % st)
    return c


def ray_minima(c) -> list:
    """The local minima on alpha > 0 of the polynomial with coefficients c
    (lowest first): the real positive roots of its derivative where the second
    derivative is positive.  The roots come from the companion matrix of the
    derivative after scaling alpha so that they lie in (0, 1] (Fujiwara's bound),
    each polished by Newton's method on the unscaled derivative."""
    c = np.asarray(c, np.float64)
    d = np.array([(k + 1) * c[k + 1] for k in range(len(c) - 1)])
    n = len(d) - 1
    while n > 0 and d[n] == 0.0:
        n -= 1
    if n < 1:
        return []
    d = d[:n + 1]
    terms = [abs(d[n - i] / d[n]) ** (1.0 / i) for i in range(1, n)]
    terms.append((abs(d[0] / d[n]) / 2.0) ** (1.0 / n))
    bound = 2.0 * max(terms)
    if not np.isfinite(bound) or bound <= 0.0:
        return []
    scaled = d * bound ** np.arange(n + 1)
    roots = np.roots(scaled[::-1]) * bound
    dd = np.array([(k + 1) * d[k + 1] for k in range(n)])
    out = []
    for z in roots:
        if abs(z.imag) > 1e-6 * abs(z) or z.real <= 0.0:
            continue
        a = float(z.real)
        for _ in range(8):  # Newton on the derivative
            fp, fpp = np.polyval(d[::-1], a), np.polyval(dd[::-1], a)
            if fpp == 0.0:
                break
            step = fp / fpp
            if not np.isfinite(step) or abs(step) > 0.5 * a:
                break
            a -= step
        if np.polyval(dd[::-1], a) > 0.0:
            out.append(a)
    return sorted(set(out))


def gd_step_exact(t: Tensor, factors, lambda_reg: float = 0.0, alpha_prev: float = 0.0):
    """GD step with the exact line search: alpha = the minimiser of
    phi(alpha) = f(theta - alpha grad) over alpha > 0 (the local minimum of the
    degree-6 polynomial phi with the smallest value of f, evaluated from the
    definition with orc_loss), taken when it lowers f; otherwise the
    backtracking step of gd_step.  Returns (status, [A,B,C] updated copies,
    alpha, loss, g2)."""
    R, F = _factors_rw(t, factors)
    G = gd_gradient(t, F, lambda_reg)
    g2 = float(sum(np.sum(g * g) for g in G))
    f0 = loss(t, F, lambda_reg)
    best, best_f = None, f0
    for a in ray_minima(gd_ray_poly(t, F, G, lambda_reg)):
        fa = loss(t, [F[m] - a * G[m] for m in range(3)], lambda_reg)
        if fa < best_f:
            best, best_f = a, fa
    if best is None:
        return gd_step(t, F, alpha_prev, lambda_reg)
    return OK, [F[m] - best * G[m] for m in range(3)], best, best_f, g2


class Ratings:
    """Observed ratings of the joint model (Appendix F): yidx int32[2, nnzY]
    (user i, item j), yval float32[nnzY]."""

    def __init__(self, yidx, yval):
        self.idx = np.ascontiguousarray(np.asarray(yidx, dtype=np.int32).reshape(2, -1))
        self.val = np.ascontiguousarray(np.asarray(yval, dtype=np.float32).reshape(-1))
        self.nnz = int(self.val.shape[0])


def joint_loss(y: Ratings, t: Tensor, factors, mu: float, lam: float) -> float:
    R = int(np.asarray(factors[0]).shape[1])
    F = [_f64(factors[m], int(t.dims[m]), R) for m in range(3)]
    return _load().orc_joint_loss(y.nnz, _p(y.idx), _p(y.val), t.nnz, _p(t.idx), _p(t.val),
                                  _p(t.dims), R, float(mu), float(lam), _p(F[0]), _p(F[1]), _p(F[2]))


def joint_gradient(y: Ratings, t: Tensor, factors, mu: float, lam: float):
    R = int(np.asarray(factors[0]).shape[1])
    F = [_f64(factors[m], int(t.dims[m]), R) for m in range(3)]
    G = [np.zeros_like(F[m]) for m in range(3)]
    st = _load().orc_joint_gradient(y.nnz, _p(y.idx), _p(y.val), t.nnz, _p(t.idx), _p(t.val),
                                    _p(t.dims), R, float(mu), float(lam), _p(F[0]), _p(F[1]),
                                    _p(F[2]), _p(G[0]), _p(G[1]), _p(G[2]))
    if st != OK:
        raise MemoryError("orc_joint_gradient status %d" % st)
    return G


def joint_als_sweep(y: Ratings, t: Tensor, factors, mu: float, lam: float):
    """Returns (status, [A,B,C] updated copies)."""
    R, F = _factors_rw(t, factors)
    st = _load().orc_joint_als_sweep(y.nnz, _p(y.idx), _p(y.val), t.nnz, _p(t.idx), _p(t.val),
                                     _p(t.dims), R, float(mu), float(lam), _p(F[0]), _p(F[1]),
                                     _p(F[2]))
    return st, F


def joint_gd_step(y: Ratings, t: Tensor, factors, mu: float, lam: float, alpha_prev: float = 0.0):
    """Returns (status, [A,B,C] updated copies, alpha, loss, g2)."""
    R, F = _factors_rw(t, factors)
    a = np.array([alpha_prev], np.float64)
    lo = np.zeros(1, np.float64)
    g2 = np.zeros(1, np.float64)
    st = _load().orc_joint_gd_step(y.nnz, _p(y.idx), _p(y.val), t.nnz, _p(t.idx), _p(t.val),
                                   _p(t.dims), R, float(mu), float(lam), _p(F[0]), _p(F[1]),
                                   _p(F[2]), _p(a), _p(lo), _p(g2))
    return st, F, float(a[0]), float(lo[0]), float(g2[0])

