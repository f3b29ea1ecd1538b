"""ctypes front end of the oracle's plain C solvers (oracle/cpcg.c): test
infrastructure and the timed CPU baseline only.

pcg: Algorithm 1 (§3.3) on a CSR matrix over `threads` OpenMP threads, the
  same iteration as oracle.pcg.pcg (one thread is the paper's one-core CPU
  baseline of §5.2).
ichol: incomplete Cholesky with a drop tolerance (§5.2, Table 2's CPU solver,
  droptol 1e-3): an entry l_ik is dropped when |l_ik| < droptol ||A(k:n,k)||_1.
pcg_ic: CG preconditioned by (L L^T)^-1, stopping on Algorithm 1's
  r^T P^-1 r so that iteration counts compare with pcg's.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import scipy.sparse as sp

from . import cbuild

_lib = None
_D = C.POINTER(C.c_double)
_LL = C.POINTER(C.c_longlong)
_I = C.POINTER(C.c_int)


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(cbuild.build())
        L.oracle_pcg.restype = C.c_int
        L.oracle_pcg.argtypes = [C.c_int, _LL, _I, _D, _D, _D, _D, C.c_double, C.c_int, C.c_int, C.c_int, _D]
        L.oracle_ichol.restype = C.c_int
        L.oracle_ichol.argtypes = [C.c_int, _LL, _I, _D, C.c_double, C.POINTER(C.c_void_p), C.POINTER(C.c_longlong)]
        L.oracle_ichol_free.restype = None
        L.oracle_ichol_free.argtypes = [C.c_void_p]
        L.oracle_ichol_export.restype = None
        L.oracle_ichol_export.argtypes = [C.c_void_p, _LL, _I, _D, _D]
        L.oracle_pcg_ic.restype = C.c_int
        L.oracle_pcg_ic.argtypes = [C.c_int, _LL, _I, _D, _D, _D, _D, C.c_void_p, C.c_double, C.c_int, _D]
        L.oracle_threads_available.restype = C.c_int
        L.oracle_threads_available.argtypes = []
        _lib = L
    return _lib


def threads_available() -> int:
    return int(lib().oracle_threads_available())


class CSR:
    """A scipy CSR matrix in the C solvers' layout (int64 row pointers, int32 columns)."""

    def __init__(self, A):
        A = sp.csr_matrix(A)
        A.sort_indices()
        self.n = A.shape[0]
        self.rp = np.ascontiguousarray(A.indptr, dtype=np.int64)
        self.ci = np.ascontiguousarray(A.indices, dtype=np.int32)
        self.v = np.ascontiguousarray(A.data, dtype=np.float64)

    def args(self):
        return (self.n, self.rp.ctypes.data_as(_LL), self.ci.ctypes.data_as(_I), self.v.ctypes.data_as(_D))


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def pcg(A, b, x0, pinv, rtol, max_iter=20000, resid_period=50, threads=1):
    """Algorithm 1 in C. Returns (x, iterations, delta_final, delta_b)."""
    M = A if isinstance(A, CSR) else CSR(A)
    b, pinv = _d(b), _d(pinv)
    x = np.array(x0, dtype=np.float64, copy=True)
    out = np.zeros(3)
    rc = lib().oracle_pcg(*M.args(), b.ctypes.data_as(_D), x.ctypes.data_as(_D), pinv.ctypes.data_as(_D),
                          float(rtol), int(max_iter), int(resid_period), int(threads), out.ctypes.data_as(_D))
    if rc != 0:
        raise MemoryError("oracle_pcg: out of memory")
    return x, int(out[0]), float(out[1]), float(out[2])


class IC:
    """Incomplete Cholesky factor L (lower triangular, L L^T ~ A)."""

    def __init__(self, A, droptol: float):
        self.A = A if isinstance(A, CSR) else CSR(A)
        h = C.c_void_p()
        nnz = C.c_longlong()
        rc = lib().oracle_ichol(*self.A.args(), float(droptol), C.byref(h), C.byref(nnz))
        if rc == 1:
            raise ArithmeticError("incomplete Cholesky: non-positive pivot")
        if rc != 0:
            raise MemoryError("incomplete Cholesky: out of memory")
        self.h, self.nnz = h, int(nnz.value)

    def matrix(self):
        """L as a scipy CSR matrix (diagonal included)."""
        n = self.A.n
        rp = np.zeros(n + 1, dtype=np.int64)
        ci = np.zeros(max(self.nnz, 1), dtype=np.int32)
        v = np.zeros(max(self.nnz, 1))
        dg = np.zeros(n)
        lib().oracle_ichol_export(self.h, rp.ctypes.data_as(_LL), ci.ctypes.data_as(_I), v.ctypes.data_as(_D),
                                  dg.ctypes.data_as(_D))
        L = sp.csr_matrix((v[: self.nnz], ci[: self.nnz], rp), shape=(n, n))
        return (L + sp.diags(dg)).tocsr()

    def close(self):
        if self.h:
            lib().oracle_ichol_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pcg_ic(A, b, x0, pinv, factor: IC, rtol, max_iter=20000):
    """CG with the (L L^T)^-1 preconditioner in C. Returns (x, iterations, r^T P^-1 r, delta_b)."""
    M = factor.A
    b, pinv = _d(b), _d(pinv)
    x = np.array(x0, dtype=np.float64, copy=True)
    out = np.zeros(3)
    rc = lib().oracle_pcg_ic(*M.args(), b.ctypes.data_as(_D), x.ctypes.data_as(_D), pinv.ctypes.data_as(_D),
                             factor.h, float(rtol), int(max_iter), out.ctypes.data_as(_D))
    if rc != 0:
        raise MemoryError("oracle_pcg_ic: out of memory")
    return x, int(out[0]), float(out[1]), float(out[2])
