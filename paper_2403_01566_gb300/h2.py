"""Thin ctypes binding of the C ABI declared in include/h2.h.

Argument marshalling only: every step of the product runs in the CUDA library
``lib/libh2gb300.so`` (built in-tree by ``__graft_entry__.build()``).  There is
no CPU fallback; loading fails loudly when the library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libh2gb300.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "h2.h")

H2_OK, H2_EINVAL, H2_ETREE, H2_ENOMEM, H2_ETIMEOUT, H2_ENOCONV, H2_ECUDA, H2_ERANK, H2_ENOTREADY = (
    0, -1, -2, -3, -4, -5, -6, -7, -8)


class BuildOpts(C.Structure):
    _fields_ = [("eta", C.c_double), ("leaf_size", C.c_int), ("order", C.c_int), ("kernel", C.c_int),
                ("kparam", C.c_double * 4), ("dim", C.c_int)]


class MulOpts(C.Structure):
    _fields_ = [("theta", C.c_double), ("max_rank", C.c_int), ("precision", C.c_int), ("sync", C.c_int),
                ("stream", C.c_void_p), ("svd_max_sweeps", C.c_int)]


class BatchOpts(C.Structure):
    _fields_ = [("test_unreachable_wait", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("n", C.c_int64), ("dim", C.c_int), ("depth", C.c_int), ("nclusters", C.c_int),
                ("nadm", C.c_int), ("ninadm", C.c_int), ("kpad", C.c_int), ("row_rank_min", C.c_int),
                ("row_rank_max", C.c_int), ("col_rank_min", C.c_int), ("col_rank_max", C.c_int),
                ("nagglomerated", C.c_int), ("device_bytes", C.c_int64), ("launches", C.c_int),
                ("workspace_bytes", C.c_int64)]


class KernelProf(C.Structure):
    _fields_ = [("launches", C.c_int), ("jobs", C.c_int), ("ms", C.c_double), ("flops", C.c_double),
                ("bytes", C.c_double)]


class H2Error(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = _lib().h2_strerror(code).decode() if _LIB is not None else str(code)
        extra = _lib().h2_last_cuda_error().decode() if _LIB is not None else ""
        super().__init__(f"{where}: {msg} ({code}) {extra}".strip())


_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
        lib = C.CDLL(LIB_PATH)
        vp, i64, dp = C.c_void_p, C.c_int64, C.POINTER(C.c_double)
        lib.h2_build.argtypes = [dp, i64, C.POINTER(BuildOpts), C.POINTER(vp)]
        lib.h2_mul.argtypes = [vp, vp, C.c_double, C.POINTER(MulOpts), C.POINTER(vp)]
        lib.h2_check.argtypes = [vp]
        lib.h2_mul_profile.argtypes = [vp, vp, C.c_double, C.POINTER(MulOpts), C.POINTER(KernelProf), C.POINTER(vp)]
        lib.h2_matvec.argtypes = [vp, vp, vp, C.c_int]
        lib.h2_matvec_batch.argtypes = [vp, vp, vp, C.c_int, C.c_int, vp]
        lib.h2_mul_h.argtypes = [vp, vp, C.c_double, C.POINTER(MulOpts), C.POINTER(vp)]
        lib.h2_hmatrix_to_dense.argtypes = [vp, vp, C.c_int]
        lib.h2_hmatrix_ranks.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                         C.POINTER(C.c_int64)]
        lib.h2_hmatrix_free.argtypes = [vp]
        lib.h2_hmatrix_free.restype = None
        lib.h2_server_create.argtypes = [C.c_int, i64, C.POINTER(vp)]
        lib.h2_server_submit.argtypes = [vp, vp, vp, C.c_double, C.POINTER(MulOpts), C.POINTER(i64)]
        lib.h2_server_wait.argtypes = [vp, i64, C.POINTER(vp), C.POINTER(C.c_double), C.POINTER(C.c_double)]
        lib.h2_server_destroy.argtypes = [vp]
        lib.h2_server_destroy.restype = None
        lib.h2_batch_create.argtypes = [C.c_int, C.POINTER(vp), C.POINTER(vp), dp, C.POINTER(MulOpts),
                                        C.POINTER(BatchOpts), C.POINTER(vp)]
        lib.h2_batch_run.argtypes = [vp, vp, C.c_int]
        lib.h2_batch_result.argtypes = [vp, C.c_int, C.POINTER(vp)]
        lib.h2_batch_info.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
        lib.h2_batch_autotune.argtypes = [vp, C.POINTER(C.c_int)]
        lib.h2_tuning_table.argtypes = [C.c_char_p, C.c_int]
        lib.h2_batch_free.argtypes = [vp]
        lib.h2_batch_free.restype = None
        lib.h2_to_dense.argtypes = [vp, vp, C.c_int]
        lib.h2_info.argtypes = [vp, C.POINTER(Stats)]
        lib.h2_ranks.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        lib.h2_permutation.argtypes = [vp, C.POINTER(C.c_int64)]
        lib.h2_free.argtypes = [vp]
        lib.h2_free.restype = None
        lib.h2_strerror.argtypes = [C.c_int]
        lib.h2_strerror.restype = C.c_char_p
        lib.h2_last_cuda_error.argtypes = []
        lib.h2_last_cuda_error.restype = C.c_char_p
        _LIB = lib
    return _LIB


def _check(rc, where):
    if rc != 0:
        raise H2Error(rc, where)


class H2Matrix:
    """Wrapper of an h2_matrix handle (owning unless owned=False: then the
    handle belongs to a batch and is never freed here)."""

    def __init__(self, handle, owned=True):
        self._h = C.c_void_p(handle)
        self._owned = owned

    @property
    def handle(self):
        return self._h

    def free(self):
        if self._h and self._h.value:
            if self._owned:
                _lib().h2_free(self._h)
            self._h = C.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def info(self) -> Stats:
        st = Stats()
        _check(_lib().h2_info(self._h, C.byref(st)), "h2_info")
        return st

    def ranks(self):
        st = self.info()
        rr = (C.c_int * st.nclusters)()
        rc = (C.c_int * st.nclusters)()
        _check(_lib().h2_ranks(self._h, rr, rc), "h2_ranks")
        return np.array(rr[:], dtype=np.int64), np.array(rc[:], dtype=np.int64)

    def permutation(self):
        st = self.info()
        p = (C.c_int64 * st.n)()
        _check(_lib().h2_permutation(self._h, p), "h2_permutation")
        return np.array(p[:], dtype=np.int64)

    def matvec(self, x):
        """y = A x for a host vector (numpy) or a CUDA torch tensor."""
        if hasattr(x, "is_cuda") and x.is_cuda:
            import torch
            y = torch.empty_like(x)
            _check(_lib().h2_matvec(self._h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), 1), "h2_matvec")
            return y
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.empty_like(x)
        _check(_lib().h2_matvec(self._h, x.ctypes.data_as(C.c_void_p), y.ctypes.data_as(C.c_void_p), 0),
               "h2_matvec")
        return y

    def matvec_batch(self, X, stream=None):
        """Y = A X for the columns of X (n x nrhs): a host numpy array, or a CUDA
        torch tensor (then Y is a CUDA tensor; the columns must be contiguous,
        i.e. X.T contiguous)."""
        if hasattr(X, "is_cuda") and X.is_cuda:
            import torch
            n, nrhs = X.shape
            Xt = X.t().contiguous()  # column-major n x nrhs
            Yt = torch.empty((nrhs, self.info().n), dtype=torch.float64, device=X.device)
            _check(_lib().h2_matvec_batch(self._h, C.c_void_p(Xt.data_ptr()), C.c_void_p(Yt.data_ptr()), nrhs, 1,
                                          C.c_void_p(stream) if stream else None), "h2_matvec_batch")
            return Yt.t()
        X = np.asarray(X, dtype=np.float64)
        n, nrhs = X.shape
        Xf = np.asfortranarray(X)
        Y = np.empty((self.info().n, nrhs), dtype=np.float64, order="F")
        _check(_lib().h2_matvec_batch(self._h, Xf.ctypes.data_as(C.c_void_p), Y.ctypes.data_as(C.c_void_p), nrhs, 0,
                                      None), "h2_matvec_batch")
        return np.ascontiguousarray(Y)

    def to_dense(self):
        st = self.info()
        out = np.empty((st.n, st.n), dtype=np.float64, order="F")
        _check(_lib().h2_to_dense(self._h, out.ctypes.data_as(C.c_void_p), 0), "h2_to_dense")
        return np.ascontiguousarray(out)

    def check(self):
        _check(_lib().h2_check(self._h), "h2_check")


def build(points, kernel, eta, leaf_size, order) -> H2Matrix:
    """h2_build on host points (n, dim) with a KernelSpec (inputs.py)."""
    pts = np.ascontiguousarray(points, dtype=np.float64)
    n, dim = pts.shape
    o = BuildOpts()
    o.eta, o.leaf_size, o.order, o.kernel, o.dim = float(eta), int(leaf_size), int(order), int(kernel.kind), int(dim)
    for i, v in enumerate(kernel.kparam()):
        o.kparam[i] = v
    h = C.c_void_p()
    _check(_lib().h2_build(pts.ctypes.data_as(C.POINTER(C.c_double)), n, C.byref(o), C.byref(h)), "h2_build")
    return H2Matrix(h.value)


def mul(A: H2Matrix, B: H2Matrix, eps: float, max_rank: int = 0, theta: float = 0.0, sync: bool = True,
        stream=None, precision: int = 0, svd_max_sweeps: int = 0) -> H2Matrix:
    """C ~ A*B with block-relative error eps (h2_mul); precision selects the
    contraction arithmetic (h2_mul_opts.precision)."""
    o = MulOpts()
    o.theta, o.max_rank, o.precision, o.sync = float(theta), int(max_rank), int(precision), 1 if sync else 0
    o.stream = stream
    o.svd_max_sweeps = int(svd_max_sweeps)
    h = C.c_void_p()
    _check(_lib().h2_mul(A.handle, B.handle, float(eps), C.byref(o), C.byref(h)), "h2_mul")
    return H2Matrix(h.value)


class HMatrix:
    """An H-matrix product (h2_mul_h): low-rank factors per admissible block,
    dense inadmissible leaves."""

    def __init__(self, handle, n_rows, n_cols):
        self._h = handle
        self.shape = (n_rows, n_cols)

    @property
    def handle(self):
        return self._h

    def ranks(self):
        na, rmax, nb = C.c_int(), C.c_int(), C.c_int64()
        _check(_lib().h2_hmatrix_ranks(self._h, None, C.byref(na), C.byref(rmax), C.byref(nb)), "h2_hmatrix_ranks")
        r = np.empty(na.value, dtype=np.int32)
        _check(_lib().h2_hmatrix_ranks(self._h, r.ctypes.data_as(C.POINTER(C.c_int)), None, None, None),
               "h2_hmatrix_ranks")
        return r

    def device_bytes(self):
        nb = C.c_int64()
        _check(_lib().h2_hmatrix_ranks(self._h, None, None, None, C.byref(nb)), "h2_hmatrix_ranks")
        return nb.value

    def to_dense(self):
        out = np.empty(self.shape, dtype=np.float64, order="F")
        _check(_lib().h2_hmatrix_to_dense(self._h, out.ctypes.data_as(C.c_void_p), 0), "h2_hmatrix_to_dense")
        return np.ascontiguousarray(out)

    def free(self):
        if self._h:
            _lib().h2_hmatrix_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def mul_h(A: H2Matrix, B: H2Matrix, eps: float, max_rank: int = 0, sync: bool = True, stream=None) -> HMatrix:
    """C ~ A*B as an H-matrix (accumulation and agglomeration, no nested-basis recompression)."""
    o = MulOpts()
    o.theta, o.max_rank, o.precision, o.sync = 0.0, int(max_rank), 0, 1 if sync else 0
    o.stream = stream
    h = C.c_void_p()
    _check(_lib().h2_mul_h(A.handle, B.handle, float(eps), C.byref(o), C.byref(h)), "h2_mul_h")
    return HMatrix(h.value, A.info().n, B.info().n)


class Server:
    """Continuous batching of products (h2_server_*): submit() returns a ticket
    at once, wait(ticket) returns (C, queued_ms, total_ms)."""

    def __init__(self, slots: int = 4, mem_budget: int = 0):
        h = C.c_void_p()
        _check(_lib().h2_server_create(int(slots), int(mem_budget), C.byref(h)), "h2_server_create")
        self._h = h.value
        self._keep = {}  # operands of requests not yet collected

    def submit(self, A: H2Matrix, B: H2Matrix, eps: float, max_rank: int = 0, precision: int = 0) -> int:
        o = MulOpts()
        o.theta, o.max_rank, o.precision, o.sync = 0.0, int(max_rank), int(precision), 1
        t = C.c_int64()
        _check(_lib().h2_server_submit(self._h, A.handle, B.handle, float(eps), C.byref(o), C.byref(t)),
               "h2_server_submit")
        self._keep[t.value] = (A, B)
        return t.value

    def wait(self, ticket: int):
        h = C.c_void_p()
        q, tot = C.c_double(), C.c_double()
        try:
            _check(_lib().h2_server_wait(self._h, int(ticket), C.byref(h), C.byref(q), C.byref(tot)), "h2_server_wait")
        finally:
            self._keep.pop(ticket, None)
        return H2Matrix(h.value), q.value, tot.value

    def close(self):
        if self._h:
            _lib().h2_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


PROFILE_KINDS = 9  # H2_PROFILE_KINDS


def mul_profile(A: H2Matrix, B: H2Matrix, eps: float, prof, max_rank: int = 0, stream=None,
                precision: int = 0) -> H2Matrix:
    """h2_mul_profile: the product with per-kernel-kind device times and work in `prof`
    (an array of PROFILE_KINDS KernelProf; kind 8 repeats the tensor-core GEMM
    stages with their tensor-core multiply-add work)."""
    if len(prof) < PROFILE_KINDS:
        raise ValueError(f"prof needs {PROFILE_KINDS} entries")
    o = MulOpts()
    o.theta, o.max_rank, o.precision, o.sync = 0.0, int(max_rank), int(precision), 1
    o.stream = stream
    h = C.c_void_p()
    _check(_lib().h2_mul_profile(A.handle, B.handle, float(eps), C.byref(o), prof, C.byref(h)), "h2_mul_profile")
    return H2Matrix(h.value)


def exported_symbols():
    """Entry points declared in include/h2.h (parsed from the header)."""
    import re
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(h2_[a-z_]+)\s*\(", text)))


class Batch:
    """Many products in merged launches (h2_batch_*): Batch([(A, B, eps), ...])
    plans them, run() replays the captured batch, result(i) is the i-th
    product (owned by the batch, overwritten by the next run)."""

    def __init__(self, products, precision=0, max_rank=0, test_unreachable_wait=False):
        self._ops = [(a, b) for a, b, _ in products]  # operands stay alive with the batch
        n = len(products)
        A = (C.c_void_p * n)(*[a.handle.value for a, _, _ in products])
        B = (C.c_void_p * n)(*[b.handle.value for _, b, _ in products])
        eps = (C.c_double * n)(*[float(e) for _, _, e in products])
        o = MulOpts()
        o.theta, o.max_rank, o.precision, o.sync = 0.0, int(max_rank), int(precision), 1
        bo = BatchOpts()
        bo.test_unreachable_wait = 1 if test_unreachable_wait else 0
        h = C.c_void_p()
        _check(_lib().h2_batch_create(n, A, B, eps, C.byref(o), C.byref(bo), C.byref(h)), "h2_batch_create")
        self._h = h
        self.n = n

    def run(self, sync=True, stream=None):
        _check(_lib().h2_batch_run(self._h, C.c_void_p(stream) if stream else None, 1 if sync else 0), "h2_batch_run")

    def result(self, i) -> H2Matrix:
        h = C.c_void_p()
        _check(_lib().h2_batch_result(self._h, int(i), C.byref(h)), "h2_batch_result")
        return H2Matrix(h.value, owned=False)

    def info(self):
        a, b, c = C.c_int(), C.c_int(), C.c_int()
        _check(_lib().h2_batch_info(self._h, C.byref(a), C.byref(b), C.byref(c)), "h2_batch_info")
        return {"launches": a.value, "chains": b.value, "kernel_launches": c.value}

    def autotune(self):
        n = C.c_int()
        _check(_lib().h2_batch_autotune(self._h, C.byref(n)), "h2_batch_autotune")
        return n.value

    def free(self):
        if self._h and self._h.value:
            _lib().h2_batch_free(self._h)
            self._h = C.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def tuning_table() -> str:
    n = _lib().h2_tuning_table(None, 0)
    buf = C.create_string_buffer(n + 1)
    _lib().h2_tuning_table(buf, n + 1)
    return buf.value.decode()
