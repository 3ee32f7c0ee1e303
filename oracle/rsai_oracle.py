"""ctypes wrapper of ``rsai_oracle.c`` plus plain NumPy pieces of the oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).  ``build_library()``
compiles the C file with gcc; nothing here touches a GPU.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

DROP_NONE, DROP_ADAPTIVE, DROP_FIXED = 0, 1, 2
FLAG_CONVERGED, FLAG_RANK, FLAG_NONFINITE = 1, 2, 4
_DROP = {"none": DROP_NONE, "adaptive": DROP_ADAPTIVE, "fixed": DROP_FIXED}

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rsai_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "librsai_oracle.so")
_lib = None
_lock = threading.Lock()

_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")


def build_library(force: bool = False) -> str:
    """Compile the oracle (gcc, OpenMP, -O2; portable flags only)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build_library())
            mat = [ctypes.c_int64, _i64p, _i32p, _f64p, _i64p, _i32p, _f64p]
            lib.ro_build.restype = ctypes.c_void_p
            lib.ro_build.argtypes = mat + [ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                           ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_int32]
            lib.ro_nnz.restype = ctypes.c_int64
            lib.ro_nnz.argtypes = [ctypes.c_void_p]
            lib.ro_export.restype = None
            lib.ro_export.argtypes = [ctypes.c_void_p, _i64p, _i32p, _f64p, _f64p, _i32p, _i32p, _f64p]
            lib.ro_free.restype = None
            lib.ro_free.argtypes = [ctypes.c_void_p]
            lib.ro_norm1.restype = ctypes.c_double
            lib.ro_norm1.argtypes = [ctypes.c_int64, _i64p, _f64p]
            lib.ro_refit.restype = None
            lib.ro_refit.argtypes = mat + [_i64p, _i32p, _f64p, _f64p, ctypes.c_int32]
            lib.ro_backward.restype = None
            lib.ro_backward.argtypes = mat + [_i64p, _i32p, _f64p, ctypes.c_void_p, _f64p]
            _lib = lib
    return _lib


def _mat(A):
    return (int(A.n), np.ascontiguousarray(A.row_ptr, np.int64), np.ascontiguousarray(A.col_idx, np.int32),
            np.ascontiguousarray(A.val, np.float64), np.ascontiguousarray(A.col_ptr, np.int64),
            np.ascontiguousarray(A.row_idx, np.int32), np.ascontiguousarray(A.cval, np.float64))


@dataclasses.dataclass
class OracleM:
    """Columns of M as built by the oracle (column-wise, rows ascending)."""

    n: int
    cols: np.ndarray  # which columns k were built (int64)
    colptr: np.ndarray  # int64[len(cols)+1]
    rows: np.ndarray  # int32[nnz]  (the pattern J_k of each column)
    vals: np.ndarray  # float64[nnz]
    rho: np.ndarray  # ||r_k||
    loops: np.ndarray  # loops l used
    flags: np.ndarray  # FLAG_* bits
    counters: np.ndarray  # [qr_flops, res_flops, bytes, solves, drops, p_max, q_max, p, sel_flops]

    @property
    def nnz(self) -> int:
        return int(self.colptr[-1])

    def column(self, t: int):
        a, b = self.colptr[t], self.colptr[t + 1]
        return self.rows[a:b], self.vals[a:b]

    def frob(self) -> float:
        """||AM - I||_F = sqrt(sum_k ||r_k||^2) (Section 2, Eq. 2.1-2.2)."""
        return float(np.sqrt(np.sum(self.rho**2)))

    def n_c(self, eps: float) -> int:
        """Columns whose residual norm stays above eps (Section 5 metric n_c)."""
        return int(np.sum(self.rho > eps))

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, len(self.cols)))
        for t in range(len(self.cols)):
            r, v = self.column(t)
            d[r, t] = v
        return d

    def csr(self):
        """Full M (all n columns built) as CSR arrays (row_ptr, col_idx, val)."""
        assert len(self.cols) == self.n and np.all(self.cols == np.arange(self.n))
        colk = np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.colptr))
        order = np.lexsort((colk, self.rows))
        row_ptr = np.zeros(self.n + 1, np.int64)
        np.add.at(row_ptr, self.rows.astype(np.int64) + 1, 1)
        return np.cumsum(row_ptr), colk[order].astype(np.int32), self.vals[order]


def build(A, c=3, l_max=10, eps=0.3, drop="fixed", tol=1e-3, tie_band=1e-12, cols=None, threads=0,
          init="identity", select="rsai") -> OracleM:
    """RSAI(tol) columns of M (Algorithm 1 + Eq. 4.3) for the given columns.
    ``init``: the initial pattern J_k^(0) of Algorithm 1, "identity" ({k})
    or "A" (the rows of column k of A).  ``select``: "rsai" (dominant rows,
    Algorithm 1) or "spai" (the c most profitable indices of Section 2,
    Eqs. 2.5-2.7), the same solve, drop and residual otherwise."""
    lib = _load()
    args = _mat(A)
    mode = _DROP[drop] if isinstance(drop, str) else int(drop)
    if cols is None:
        colsa = np.arange(A.n, dtype=np.int64)
        ptr = None
    else:
        colsa = np.ascontiguousarray(cols, dtype=np.int64)
        ptr = colsa.ctypes.data_as(ctypes.c_void_p)
    h = lib.ro_build(*args, int(c), int(l_max), float(eps), mode, float(tol), float(tie_band),
                     ptr, int(len(colsa)), int(threads), {"identity": 0, "A": 1}[init],
                     {"rsai": 0, "spai": 1}[select])
    try:
        nnz = lib.ro_nnz(h)
        nc = len(colsa)
        colptr = np.zeros(nc + 1, np.int64)
        rows = np.zeros(max(nnz, 1), np.int32)
        vals = np.zeros(max(nnz, 1), np.float64)
        rho = np.zeros(max(nc, 1))
        loops = np.zeros(max(nc, 1), np.int32)
        flags = np.zeros(max(nc, 1), np.int32)
        counters = np.zeros((max(nc, 1), 9))
        lib.ro_export(h, colptr, rows, vals, rho, loops, flags, counters)
    finally:
        lib.ro_free(h)
    return OracleM(n=int(A.n), cols=colsa, colptr=colptr, rows=rows[:nnz], vals=vals[:nnz],
                   rho=rho[:nc], loops=loops[:nc], flags=flags[:nc], counters=counters[:nc])


def norm1(A) -> float:
    """||A||_1, the maximum column absolute sum (Eq. 4.3)."""
    return float(_load().ro_norm1(int(A.n), np.ascontiguousarray(A.col_ptr, np.int64),
                                  np.ascontiguousarray(A.cval, np.float64)))


def refit(A, colptr, rows, threads=0):
    """Frozen-pattern LS re-solve (Eq. 2.3); returns (M values, rho_k^2)."""
    lib = _load()
    vals = np.zeros(max(int(colptr[-1]), 1))
    rho2 = np.zeros(int(A.n))
    lib.ro_refit(*_mat(A), np.ascontiguousarray(colptr, np.int64), np.ascontiguousarray(rows, np.int32),
                 vals, rho2, int(threads))
    return vals[: int(colptr[-1])], rho2


def backward(A, colptr, rows, grad_m, grad_rho2=None):
    """dL/d(values of A) in CSR order through every frozen-pattern LS solve."""
    lib = _load()
    out = np.zeros(A.nnz if hasattr(A, "nnz") else int(A.row_ptr[-1]))
    gm = np.ascontiguousarray(grad_m, np.float64)
    if gm.size == 0:
        gm = np.zeros(1)
    gr = None if grad_rho2 is None else np.ascontiguousarray(grad_rho2, np.float64)
    lib.ro_backward(*_mat(A), np.ascontiguousarray(colptr, np.int64), np.ascontiguousarray(rows, np.int32),
                    gm, None if gr is None else gr.ctypes.data_as(ctypes.c_void_p), out)
    return out


def spmv(row_ptr, col_idx, val, x):
    """y = A x for CSR arrays (plain NumPy)."""
    n = len(row_ptr) - 1
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    return np.bincount(rows, weights=np.asarray(val) * np.asarray(x)[col_idx], minlength=n)


@dataclasses.dataclass
class SolveResult:
    x: np.ndarray
    iters: int
    converged: bool
    relres_true: float
    status: str


def bicgstab(A, M=None, b=None, rtol=1e-8, maxit=1000) -> SolveResult:
    """Right-preconditioned BiCGStab on A M y = b, x = M y (Eq. 1.2; Section 5).

    x0 = 0.  Textbook BiCGStab (van der Vorst) on the operator A M.  The
    recursive residual is tested after the half step (s) and the full step (r);
    an exit at the half step counts as the full iteration it belongs to.  On
    exit the true residual ||b - A x|| / ||b|| is reported.  ``M`` is a CSR
    triple (row_ptr, col_idx, val) or None for no preconditioner.
    """
    def Aop(v):
        return spmv(A.row_ptr, A.col_idx, A.val, v)

    def Mop(v):
        return v if M is None else spmv(M[0], M[1], M[2], v)

    n = int(A.n)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    y = np.zeros(n)
    r = b.copy()
    rhat = r.copy()
    rho_old = alpha = omega = 1.0
    v = np.zeros(n)
    p = np.zeros(n)
    status = "maxit"
    it = 0
    if nb == 0.0:
        return SolveResult(np.zeros(n), 0, True, 0.0, "converged")
    for it in range(1, maxit + 1):
        rho = float(rhat @ r)
        if rho == 0.0:
            status = "breakdown_rho"
            break
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = Aop(Mop(p))
        rv = float(rhat @ v)
        if rv == 0.0:  # alpha = rho / (rhat^T v) is undefined
            status = "breakdown_alpha"
            break
        alpha = rho / rv
        s = r - alpha * v
        if np.linalg.norm(s) / nb < rtol:
            y = y + alpha * p
            status = "converged"
            break
        t = Aop(Mop(s))
        tt = float(t @ t)
        if tt == 0.0:
            status = "breakdown_omega"
            break
        omega = float(t @ s) / tt
        y = y + alpha * p + omega * s
        r = s - omega * t
        if np.linalg.norm(r) / nb < rtol:
            status = "converged"
            break
        if omega == 0.0:
            status = "breakdown_omega"
            break
        rho_old = rho
    x = Mop(y)
    rel = float(np.linalg.norm(b - Aop(x)) / nb)
    return SolveResult(x, it, status == "converged", rel, status)
