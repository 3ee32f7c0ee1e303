"""Python binding of the C ABI in ``include/rsai.h`` (ctypes; argument marshalling only).

Every step of RSAI(tol) runs in the CUDA kernels of ``librsai.so``; this module
only passes pointers, sizes and the current CUDA stream.  PyTorch provides the
device memory of inputs and outputs.  There is no CPU fallback: if the library
is missing or no GPU is visible, calls raise.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librsai.so")

RSAI_OK = 0
STATUS_NAMES = {
    0: "OK", 1: "INVALID_ARG", 2: "SHAPE", 3: "UNSORTED", 4: "INDEX_RANGE", 5: "EMPTY_COLUMN", 6: "OOM",
    7: "CUDA", 8: "TIMEOUT", 9: "WORKSPACE", 10: "BREAKDOWN", 11: "NOT_CONVERGED", 12: "NO_DEVICE",
    13: "TOO_LARGE",
}
FLAG_INIT_PATTERN_A = 2  # RSAI_FLAG_INIT_PATTERN_A
FLAG_SELECT_SPAI = 4  # RSAI_FLAG_SELECT_SPAI
DROP = {"none": 0, "adaptive": 1, "fixed": 2}
PRECISION = {"fp64": 0, "fp32_refine": 1}
COL_CONVERGED, COL_RANK, COL_NONFINITE, COL_FAILED = 1, 2, 4, 8
PHASES = ("setup", "bin_warp", "bin_cta", "bin_global", "assemble")

# every symbol include/rsai.h declares
EXPORTS = [
    "rsai_abi_version", "rsai_status_string", "rsai_params_default", "rsai_params_check", "rsai_build",
    "rsai_rebuild", "rsai_set_values", "rsai_get_stats", "rsai_get_M", "rsai_get_columns", "rsai_refit",
    "rsai_apply", "rsai_backward", "rsai_bicgstab", "rsai_handle_free", "rsai_peak_fma", "rsai_build_phase_times",
    "rsai_bicgstab_noalloc", "rsai_build_batch", "rsai_get_block_stats", "rsai_get_tuning", "rsai_set_tuning",
    "rsai_set_allocator", "rsai_get_M_csc", "rsai_spmv", "rsai_spmv_grad_values",
]


class RSAIError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: RSAI status {status} ({STATUS_NAMES.get(status, '?')}): {status_string(status)}")


class CSR(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("row_ptr", ctypes.c_void_p),
                ("col_idx", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class CSC(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("col_ptr", ctypes.c_void_p),
                ("row_idx", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class Params(ctypes.Structure):
    _fields_ = [("c", ctypes.c_int32), ("l_max", ctypes.c_int32), ("eps", ctypes.c_double),
                ("drop_mode", ctypes.c_int32), ("tol", ctypes.c_double), ("precision", ctypes.c_int32),
                ("tie_band", ctypes.c_double), ("flags", ctypes.c_uint32)]


class Tuning(ctypes.Structure):
    _fields_ = [("warp_bin_warps", ctypes.c_int32), ("warp_bin_ctas_per_sm", ctypes.c_int32),
                ("small_qr_max_p", ctypes.c_int32), ("global_bin_ctas", ctypes.c_int32), ("half_bin", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class Stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz_A", ctypes.c_int64), ("nnz_M", ctypes.c_int64),
                ("n_c", ctypes.c_int64), ("frob", ctypes.c_double), ("norm1_A", ctypes.c_double),
                ("qr_flops", ctypes.c_double), ("res_flops", ctypes.c_double), ("refine_flops", ctypes.c_double),
                ("refine_flops_f64", ctypes.c_double),
                ("bytes", ctypes.c_double), ("loops", ctypes.c_int64), ("solves", ctypes.c_int64),
                ("drops", ctypes.c_int64), ("p_max", ctypes.c_int32), ("q_max", ctypes.c_int32),
                ("cols_bin", ctypes.c_int64 * 3), ("n_rank", ctypes.c_int64), ("n_nonfinite", ctypes.c_int64),
                ("n_failed", ctypes.c_int64), ("cols_bin_half", ctypes.c_int64), ("select_flops", ctypes.c_double)]

    def as_dict(self) -> dict:
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            d[name] = list(v) if name == "cols_bin" else v
        return d


# device allocator callbacks (rsai_alloc_fn / rsai_free_fn)
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)

_lib = None
_allocators = []  # every callback pair ever installed (handles keep calling theirs until freed)


def load(build_if_missing: bool = False):
    """Load librsai.so (raises if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        if build_if_missing:
            from . import build_ext

            build_ext.build()
        else:
            raise RuntimeError(f"librsai.so is not built ({LIB_PATH}); run paper_1503_04500_gb300/build_ext.py")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "rsai_abi_version": (i32, []),
        "rsai_status_string": (ctypes.c_char_p, [i32]),
        "rsai_params_default": (i32, [ctypes.POINTER(Params)]),
        "rsai_params_check": (i32, [ctypes.POINTER(Params)]),
        "rsai_build": (i32, [ctypes.POINTER(CSR), ctypes.POINTER(CSC), ctypes.POINTER(Params), vp,
                             ctypes.POINTER(vp)]),
        "rsai_rebuild": (i32, [vp, vp]),
        "rsai_set_values": (i32, [vp, vp, vp]),
        "rsai_get_stats": (i32, [vp, vp, ctypes.POINTER(Stats)]),
        "rsai_get_M": (i32, [vp, vp, vp, vp, vp]),
        "rsai_get_columns": (i32, [vp, vp, vp, vp, vp]),
        "rsai_refit": (i32, [vp, vp, vp, vp, vp]),
        "rsai_apply": (i32, [vp, vp, vp, vp]),
        "rsai_backward": (i32, [vp, vp, vp, vp, vp, vp]),
        "rsai_bicgstab": (i32, [ctypes.POINTER(CSR), vp, vp, vp, f64, i32, ctypes.POINTER(i32),
                                ctypes.POINTER(f64), vp]),
        "rsai_handle_free": (None, [vp]),
        "rsai_peak_fma": (i32, [i32, vp, ctypes.POINTER(f64)]),
        "rsai_build_phase_times": (i32, [vp, vp, ctypes.POINTER(f64)]),
        "rsai_build_batch": (i32, [ctypes.POINTER(CSR), ctypes.POINTER(CSC), i32, ctypes.POINTER(Params), vp,
                                   ctypes.POINTER(vp)]),
        "rsai_get_block_stats": (i32, [vp, vp, vp, vp, vp]),
        "rsai_get_tuning": (i32, [vp, ctypes.POINTER(Tuning)]),
        "rsai_set_tuning": (i32, [vp, ctypes.POINTER(Tuning)]),
        "rsai_bicgstab_noalloc": (i32, [ctypes.POINTER(CSR), ctypes.POINTER(CSR), vp, vp, f64, i32,
                                        ctypes.POINTER(i32), ctypes.POINTER(f64), vp]),
        "rsai_set_allocator": (i32, [ALLOC_FN, FREE_FN, vp]),
        "rsai_get_M_csc": (i32, [vp, vp, vp, vp, vp]),
        "rsai_spmv": (i32, [ctypes.POINTER(CSR), vp, vp, vp]),
        "rsai_spmv_grad_values": (i32, [ctypes.POINTER(CSR), vp, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def use_torch_allocator() -> None:
    """Take the library's device memory from PyTorch's caching allocator.

    Applies to handles created afterwards (each handle frees with the
    allocator it was created with), to refit temporaries and to the BiCGStab
    workspace.  The callbacks run on the calling thread, outside any graph
    replay.
    """
    import torch

    def _alloc(nbytes, stream, ctx):
        return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), int(stream or 0))

    def _free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    cbs = (ALLOC_FN(_alloc), FREE_FN(_free))
    _allocators.append(cbs)
    _check(load().rsai_set_allocator(cbs[0], cbs[1], None), "rsai_set_allocator")


def use_cuda_allocator() -> None:
    """Restore cudaMallocAsync / cudaFreeAsync for handles created afterwards.

    The earlier callbacks stay referenced: handles created under them still
    free through them.
    """
    _check(load().rsai_set_allocator(ALLOC_FN(), FREE_FN(), None), "rsai_set_allocator")


def status_string(status: int) -> str:
    return load().rsai_status_string(int(status)).decode()


def _check(status: int, where: str, ok=(RSAI_OK,)):
    if status not in ok:
        raise RSAIError(status, where)
    return status


def _stream(stream=None):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t) -> int:
    """Address of a torch tensor or a contiguous numpy array (host)."""
    if isinstance(t, np.ndarray):
        assert t.flags["C_CONTIGUOUS"]
        return t.ctypes.data
    assert t.is_contiguous()
    return t.data_ptr()


def default_params(**kw) -> Params:
    p = Params()
    _check(load().rsai_params_default(ctypes.byref(p)), "rsai_params_default")
    for k, v in kw.items():
        if k == "drop":
            p.drop_mode = DROP[v] if isinstance(v, str) else int(v)
        elif k == "precision":
            p.precision = PRECISION[v] if isinstance(v, str) else int(v)
        elif k == "init":
            # initial pattern J_k^(0) (Algorithm 1): "identity" ({k}) or "A" (rows of A(:,k))
            p.flags = (p.flags & ~FLAG_INIT_PATTERN_A) | (FLAG_INIT_PATTERN_A if v == "A" else 0)
        elif k == "select":
            # new indices: "rsai" (dominant rows, Algorithm 1) or "spai" (most profitable, Eqs. 2.5-2.7)
            p.flags = (p.flags & ~FLAG_SELECT_SPAI) | (FLAG_SELECT_SPAI if v == "spai" else 0)
        else:
            setattr(p, k, v)
    return p


@dataclasses.dataclass
class DeviceMatrix:
    """A in CSR + CSC as torch tensors (device or pinned/host)."""

    n: int
    nnz: int
    row_ptr: object
    col_idx: object
    val: object
    col_ptr: object
    row_idx: object
    cval: object

    @classmethod
    def from_host(cls, A, device="cuda"):
        import torch

        t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a, dtype=dt)).to(device)  # noqa: E731
        return cls(int(A.n), int(A.nnz), t(A.row_ptr, np.int64), t(A.col_idx, np.int32), t(A.val, np.float64),
                   t(A.col_ptr, np.int64), t(A.row_idx, np.int32), t(A.cval, np.float64))

    def csr(self) -> CSR:
        return CSR(self.n, self.nnz, _ptr(self.row_ptr), _ptr(self.col_idx), _ptr(self.val))

    def csc(self) -> CSC:
        return CSC(self.n, self.nnz, _ptr(self.col_ptr), _ptr(self.row_idx), _ptr(self.cval))


def _host_structs(A):
    """CSR/CSC structs over host (numpy) arrays of a SparseMatrix-like object."""
    keep = [np.ascontiguousarray(A.row_ptr, np.int64), np.ascontiguousarray(A.col_idx, np.int32),
            np.ascontiguousarray(A.val, np.float64), np.ascontiguousarray(A.col_ptr, np.int64),
            np.ascontiguousarray(A.row_idx, np.int32), np.ascontiguousarray(A.cval, np.float64)]
    csr = CSR(int(A.n), int(keep[1].size), keep[0].ctypes.data, keep[1].ctypes.data, keep[2].ctypes.data)
    csc = CSC(int(A.n), int(keep[4].size), keep[3].ctypes.data, keep[4].ctypes.data, keep[5].ctypes.data)
    return csr, csc, keep


class Handle:
    """A built M (owned by the library until ``free``)."""

    def __init__(self, ptr: int, n: int, params: Params, status: int):
        self._h = ctypes.c_void_p(ptr)
        self.n = n
        self.params = params
        self.status = status

    def __del__(self):
        self.free()

    def free(self):
        if getattr(self, "_h", None) and self._h.value:
            load().rsai_handle_free(self._h)
            self._h = ctypes.c_void_p(0)

    def stats(self, stream=None) -> dict:
        s = Stats()
        st = load().rsai_get_stats(self._h, _stream(stream), ctypes.byref(s))
        _check(st, "rsai_get_stats", ok=(RSAI_OK, 9))
        d = s.as_dict()
        d["status"] = st
        return d

    def M(self, stream=None):
        """M in CSR as torch cuda tensors (row_ptr int64, col_idx int32, val float64)."""
        import torch

        nnz = self.stats(stream)["nnz_M"]
        rp = torch.empty(self.n + 1, dtype=torch.int64, device="cuda")
        ci = torch.empty(max(nnz, 1), dtype=torch.int32, device="cuda")
        va = torch.empty(max(nnz, 1), dtype=torch.float64, device="cuda")
        _check(load().rsai_get_M(self._h, _ptr(rp), _ptr(ci), _ptr(va), _stream(stream)), "rsai_get_M")
        return rp, ci[:nnz], va[:nnz]

    def M_csc(self, stream=None):
        """M's pattern in CSC as torch cuda tensors: (col_ptr int64, row_idx int32,
        csc_to_csr int64), the last giving each CSC entry's position in M's CSR values."""
        import torch

        nnz = self.stats(stream)["nnz_M"]
        cp = torch.empty(self.n + 1, dtype=torch.int64, device="cuda")
        ri = torch.empty(max(nnz, 1), dtype=torch.int32, device="cuda")
        pos = torch.empty(max(nnz, 1), dtype=torch.int64, device="cuda")
        _check(load().rsai_get_M_csc(self._h, _ptr(cp), _ptr(ri), _ptr(pos), _stream(stream)), "rsai_get_M_csc")
        return cp, ri[:nnz], pos[:nnz]

    def M_host(self, nnz=None, out=None, stream=None):
        """M in CSR copied straight into host numpy arrays (one D2H copy each)."""
        if nnz is None:
            nnz = self.stats(stream)["nnz_M"]
        if out is None:
            out = (np.empty(self.n + 1, np.int64), np.empty(max(nnz, 1), np.int32), np.empty(max(nnz, 1)))
        rp, ci, va = out
        _check(load().rsai_get_M(self._h, _ptr(rp), _ptr(ci), _ptr(va), _stream(stream)), "rsai_get_M")
        return rp, ci[:nnz], va[:nnz]

    def columns(self, stream=None):
        import torch

        rho = torch.empty(self.n, dtype=torch.float64, device="cuda")
        loops = torch.empty(self.n, dtype=torch.int32, device="cuda")
        flags = torch.empty(self.n, dtype=torch.int32, device="cuda")
        _check(load().rsai_get_columns(self._h, _ptr(rho), _ptr(loops), _ptr(flags), _stream(stream)),
               "rsai_get_columns")
        return rho, loops, flags

    def block_stats(self, count: int, stream=None):
        """Per-member (||A_b M_b - I||_F, n_c, nnz(M_b)) of a batch handle."""
        frob = np.zeros(count)
        nc = np.zeros(count, np.int64)
        nz = np.zeros(count, np.int64)
        _check(load().rsai_get_block_stats(self._h, _stream(stream), _ptr(frob), _ptr(nc), _ptr(nz)),
               "rsai_get_block_stats")
        return frob, nc, nz

    def tuning(self) -> dict:
        t = Tuning()
        _check(load().rsai_get_tuning(self._h, ctypes.byref(t)), "rsai_get_tuning")
        return t.as_dict()

    def set_tuning(self, **kw):
        """rsai_set_tuning: launch shapes of the bins (CTA shapes: identical results; the
        register-QR threshold: the same solutions up to rounding)."""
        t = Tuning(**{**self.tuning(), **kw})
        _check(load().rsai_set_tuning(self._h, ctypes.byref(t)), "rsai_set_tuning")

    def rebuild(self, stream=None):
        _check(load().rsai_rebuild(self._h, _stream(stream)), "rsai_rebuild")

    def phase_times(self, stream=None):
        """Run the build once more phase by phase; per-phase milliseconds (CUDA events)."""
        ms = (ctypes.c_double * 5)()
        _check(load().rsai_build_phase_times(self._h, _stream(stream), ms), "rsai_build_phase_times")
        return dict(zip(PHASES, list(ms)))

    def set_values(self, val, stream=None):
        _check(load().rsai_set_values(self._h, _ptr(val), _stream(stream)), "rsai_set_values")

    def apply(self, x, y=None, stream=None):
        import torch

        if y is None:
            y = torch.empty_like(x)
        _check(load().rsai_apply(self._h, _ptr(x), _ptr(y), _stream(stream)), "rsai_apply")
        return y

    def refit(self, A_val, stream=None):
        """rsai_refit: (values of M in its CSR order, rho_k^2) on the frozen pattern."""
        import torch

        nnz = self.stats(stream)["nnz_M"]
        mv = torch.empty(max(nnz, 1), dtype=torch.float64, device="cuda")
        rho2 = torch.empty(self.n, dtype=torch.float64, device="cuda")
        _check(load().rsai_refit(self._h, _ptr(A_val), _ptr(mv), _ptr(rho2), _stream(stream)), "rsai_refit")
        return mv[:nnz], rho2

    def backward(self, A_val, grad_M, grad_rho2=None, stream=None):
        """rsai_backward: dL/d(values of A) for dL/dM (CSR order of M) and dL/d(rho_k^2)."""
        import torch

        g = torch.empty_like(A_val)
        _check(load().rsai_backward(self._h, _ptr(A_val), _ptr(grad_M),
                                    None if grad_rho2 is None else _ptr(grad_rho2), _ptr(g), _stream(stream)),
               "rsai_backward")
        return g


def build(A, c=3, l_max=10, eps=0.3, drop="fixed", tol=1e-3, precision="fp64", tie_band=1e-12, stream=None,
          allow_failed=False, init="identity", select="rsai") -> Handle:
    """rsai_build on a DeviceMatrix (device tensors) or a SparseMatrix-like
    object with numpy arrays (then the library copies from host memory)."""
    lib = load()
    params = default_params(c=c, l_max=l_max, eps=eps, drop=drop, tol=tol, precision=precision, tie_band=tie_band,
                            init=init, select=select)
    if isinstance(A, DeviceMatrix):
        csr, csc, keep = A.csr(), A.csc(), None
    else:
        csr, csc, keep = _host_structs(A)
    out = ctypes.c_void_p(0)
    st = lib.rsai_build(ctypes.byref(csr), ctypes.byref(csc), ctypes.byref(params), _stream(stream),
                        ctypes.byref(out))
    del keep
    ok = (RSAI_OK, 9) if allow_failed else (RSAI_OK,)
    if st not in ok:
        if out.value:
            lib.rsai_handle_free(out)
        raise RSAIError(st, "rsai_build")
    return Handle(out.value, int(csr.n), params, st)


def transpose(A):
    """A^T with no arithmetic: A's CSC arrays are the CSR of A^T and its CSR
    arrays the CSC.  Works on a DeviceMatrix (tensors shared, not copied) and
    on a SparseMatrix-like host object (its csc_to_csr map is inverted)."""
    if isinstance(A, DeviceMatrix):
        return DeviceMatrix(A.n, A.nnz, A.col_ptr, A.row_idx, A.cval, A.row_ptr, A.col_idx, A.val)
    inv = np.empty_like(A.csc_to_csr)
    inv[A.csc_to_csr] = np.arange(A.csc_to_csr.size, dtype=A.csc_to_csr.dtype)
    return dataclasses.replace(A, row_ptr=A.col_ptr, col_idx=A.row_idx, val=A.cval, col_ptr=A.row_ptr,
                               row_idx=A.col_idx, cval=A.val, csc_to_csr=inv)


class LeftHandle:
    """A left sparse approximate inverse, M A ~ I, kept as the right inverse
    M_R of A^T built by the same kernels (||M A - I||_F = ||A^T M_R - I||_F,
    and the column problems of A^T are the row problems of M).  ``right`` is
    the handle of M_R; M = M_R^T is read through M_R's CSC pattern."""

    def __init__(self, right: Handle):
        self.right = right
        self.n = right.n

    def M(self, stream=None):
        """M = M_R^T in CSR (torch cuda tensors): M_R's CSC arrays, values gathered through csc_to_csr."""
        _, _, va = self.right.M(stream)
        cp, ri, pos = self.right.M_csc(stream)
        return cp, ri, va[pos].contiguous()

    def stats(self, stream=None):
        """Statistics of M_R (frob = ||A^T M_R - I||_F = ||M A - I||_F)."""
        return self.right.stats(stream)

    def columns(self, stream=None):
        """Per row k of M: ||e_k^T - m_k^T A||, loops and flags (those of column k of M_R)."""
        return self.right.columns(stream)

    def free(self):
        self.right.free()


def build_left(A, **kw) -> LeftHandle:
    """rsai_build on A^T: a left preconditioner M with M A ~ I (same parameters as ``build``)."""
    return LeftHandle(build(transpose(A), **kw))


def build_batch(members, c=3, l_max=10, eps=0.3, drop="fixed", tol=1e-3, precision="fp64", tie_band=1e-12,
                stream=None, allow_failed=False) -> Handle:
    """rsai_build_batch over a list of DeviceMatrix (device tensors) or
    SparseMatrix-like (numpy, host) members; returns one handle whose M is
    block diagonal."""
    lib = load()
    params = default_params(c=c, l_max=l_max, eps=eps, drop=drop, tol=tol, precision=precision, tie_band=tie_band)
    csrs = (CSR * len(members))()
    cscs = (CSC * len(members))()
    keep = []
    n = 0
    for b, A in enumerate(members):
        if isinstance(A, DeviceMatrix):
            csrs[b], cscs[b] = A.csr(), A.csc()
        else:
            r, cc, k = _host_structs(A)
            csrs[b], cscs[b] = r, cc
            keep.append(k)
        n += int(csrs[b].n)
    out = ctypes.c_void_p(0)
    st = lib.rsai_build_batch(csrs, cscs, len(members), ctypes.byref(params), _stream(stream), ctypes.byref(out))
    del keep
    ok = (RSAI_OK, 9) if allow_failed else (RSAI_OK,)
    if st not in ok:
        if out.value:
            lib.rsai_handle_free(out)
        raise RSAIError(st, "rsai_build_batch")
    return Handle(out.value, n, params, st)


def bicgstab(A: DeviceMatrix, M: Handle | None, b, rtol=1e-8, maxit=1000, stream=None):
    """Right-preconditioned BiCGStab (Eq. 1.2); returns (x, iters, relres, status)."""
    import torch

    x = torch.empty_like(b)
    it = ctypes.c_int32(0)
    rr = ctypes.c_double(0.0)
    csr = A.csr()
    st = load().rsai_bicgstab(ctypes.byref(csr), None if M is None else M._h, _ptr(b), _ptr(x), float(rtol),
                              int(maxit), ctypes.byref(it), ctypes.byref(rr), _stream(stream))
    _check(st, "rsai_bicgstab", ok=(RSAI_OK, 10, 11))
    return x, it.value, rr.value, st


def bicgstab_noalloc(A: DeviceMatrix, M_csr, b, x, rtol=1e-8, maxit=1000, stream=None):
    """rsai_bicgstab_noalloc: the same solve with no device allocation (n <= 65536).

    ``M_csr`` is (row_ptr, col_idx, val) device tensors or None; ``x`` is a
    caller-owned device output.  Returns (iters, relres, status).
    """
    it = ctypes.c_int32(0)
    rr = ctypes.c_double(0.0)
    csr = A.csr()
    mcsr = None
    if M_csr is not None:
        rp, ci, va = M_csr
        mcsr = CSR(A.n, int(va.numel()), _ptr(rp), _ptr(ci), _ptr(va))
    st = load().rsai_bicgstab_noalloc(ctypes.byref(csr), None if mcsr is None else ctypes.byref(mcsr), _ptr(b),
                                      _ptr(x), float(rtol), int(maxit), ctypes.byref(it), ctypes.byref(rr),
                                      _stream(stream))
    _check(st, "rsai_bicgstab_noalloc", ok=(RSAI_OK, 10, 11))
    return it.value, rr.value, st


def spmv(row_ptr, col_idx, val, x, y=None, stream=None):
    """rsai_spmv: y = A x for A in CSR (device tensors); returns y."""
    import torch

    if y is None:
        y = torch.empty(row_ptr.numel() - 1, dtype=torch.float64, device=x.device)
    csr = CSR(row_ptr.numel() - 1, col_idx.numel(), _ptr(row_ptr), _ptr(col_idx), _ptr(val))
    _check(load().rsai_spmv(ctypes.byref(csr), _ptr(x), _ptr(y), _stream(stream)), "rsai_spmv")
    return y


def spmv_grad_values(row_ptr, col_idx, gy, x, gval=None, stream=None):
    """rsai_spmv_grad_values: gval[e] = gy[row(e)] * x[col(e)] in CSR order; returns gval."""
    import torch

    if gval is None:
        gval = torch.empty(col_idx.numel(), dtype=torch.float64, device=x.device)
    csr = CSR(row_ptr.numel() - 1, col_idx.numel(), _ptr(row_ptr), _ptr(col_idx), None)
    _check(load().rsai_spmv_grad_values(ctypes.byref(csr), _ptr(gy), _ptr(x), _ptr(gval), _stream(stream)),
           "rsai_spmv_grad_values")
    return gval


def peak_fma(fp64: bool, stream=None) -> float:
    v = ctypes.c_double(0.0)
    _check(load().rsai_peak_fma(1 if fp64 else 0, _stream(stream), ctypes.byref(v)), "rsai_peak_fma")
    return v.value
