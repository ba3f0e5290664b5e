"""Python binding of librtproj (randomized orthogonal projection on GB300).

Argument marshalling only: every step of the method runs in the CUDA kernels of
``librtproj.so`` behind the C ABI declared in ``include/rtproj.h``. PyTorch supplies
device memory (the caller-owned workspace and outputs) and the CUDA stream. There is
no CPU fallback: if the library is missing this module raises on first use.

    >>> P = Projector(A)                 # A: cuda float64 or float32, m x n, row-major
    >>> P.precondition(seed=1, l=4 * m)  # sketch, pivoted QR, Gram, Cholesky
    >>> Z = P.null_project(B)            # B: k x n (each row a right-hand side), A's dtype
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import _build

__all__ = ["Projector", "SparseProjector", "RtprojError", "load_library", "library_path", "STATUS", "MODES", "OMEGAS",
           "generate_omega", "launch_count"]

MODES = {"fp64": 0, "mixed": 1}
OMEGAS = {"uniform": 0, "rademacher": 1, "gaussian": 2}
DTYPES = {torch.float64: 0, torch.float32: 1}
STATUS = {
    0: "RTPROJ_OK", 1: "RTPROJ_EINVAL", 2: "RTPROJ_ESTATE", 3: "RTPROJ_ERANK", 4: "RTPROJ_ENOTSPD",
    5: "RTPROJ_ENONFINITE", 6: "RTPROJ_ETIMEOUT", 7: "RTPROJ_ENOMEM", 8: "RTPROJ_ECUDA", 9: "RTPROJ_EUNSUPPORTED",
}


class RtprojError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = int(code)
        super().__init__(f"{where}: {STATUS.get(self.code, self.code)}")


class Opts(ctypes.Structure):
    _fields_ = [
        ("mode", ctypes.c_int), ("omega", ctypes.c_int), ("sketch_slices", ctypes.c_int),
        ("gram_slices", ctypes.c_int), ("gram2_slices", ctypes.c_int), ("apply_slices", ctypes.c_int),
        ("resid_slices", ctypes.c_int), ("refine_passes", ctypes.c_int), ("timing", ctypes.c_int),
        ("rank_tol", ctypes.c_double), ("dtype", ctypes.c_int), ("spin_limit_cycles", ctypes.c_longlong),
        ("refine_tol", ctypes.c_double), ("scalable", ctypes.c_int), ("qr_form", ctypes.c_int),
        ("async_", ctypes.c_int),   # async_: opts.async
    ]


class Info(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int), ("preconditioned", ctypes.c_int), ("m", ctypes.c_int64), ("n", ctypes.c_int64),
        ("l", ctypes.c_int64), ("r11", ctypes.c_double), ("rmm", ctypes.c_double), ("l11", ctypes.c_double),
        ("lmm", ctypes.c_double), ("ms_precondition", ctypes.c_float), ("kappa_R", ctypes.c_double),
        ("kappa_pre", ctypes.c_double), ("norm_A", ctypes.c_double), ("resid_rel", ctypes.c_double),
        ("dh_rel", ctypes.c_double), ("passes", ctypes.c_int),
    ]


_lib = None
_P = ctypes.c_void_p
_I64 = ctypes.c_int64

EXPORTS = {
    "rtproj_default_opts": (None, [ctypes.POINTER(Opts)]),
    "rtproj_workspace_bytes": (ctypes.c_size_t, [_I64, _I64, _I64, _I64, ctypes.POINTER(Opts)]),
    "rtproj_create": (ctypes.c_int, [ctypes.POINTER(_P), _I64, _I64, _P, _I64, _I64, _I64, _P, ctypes.c_size_t, _P,
                                     ctypes.POINTER(Opts)]),
    "rtproj_precondition": (ctypes.c_int, [_P, ctypes.c_uint64, _I64]),
    "rtproj_null_project": (ctypes.c_int, [_P, _P, _I64, _I64, _P, _I64]),
    "rtproj_row_project": (ctypes.c_int, [_P, _P, _I64, _I64, _P, _I64]),
    "rtproj_lstsq": (ctypes.c_int, [_P, _P, _I64, _I64, _P, _I64]),
    "rtproj_project": (ctypes.c_int, [_P, _P, _I64, _I64, _P, _I64, _P, _I64, _P, _I64]),
    "rtproj_sketch": (ctypes.c_int, [_P, ctypes.c_uint64, _I64, _P, _I64]),
    "rtproj_export_state": (ctypes.c_int, [_P, _P, _P, _P]),
    "rtproj_get_info": (ctypes.c_int, [_P, ctypes.POINTER(Info)]),
    "rtproj_clear_status": (ctypes.c_int, [_P]),
    "rtproj_destroy": (ctypes.c_int, [_P]),
    "rtproj_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "rtproj_get_timings": (ctypes.c_int, [_P, _P, _P]),
    "rtproj_launch_count": (ctypes.c_uint64, []),
    "rtproj_sketch_noalloc": (ctypes.c_int, [_P, _I64, _I64, _I64, ctypes.c_uint64, _I64, ctypes.c_int, _P, _I64, _P]),
    "rtproj_generate_omega": (ctypes.c_int, [ctypes.c_uint64, _I64, _I64, ctypes.c_int, _P, _I64, _P]),
    "rtproj_set_spin_limit": (ctypes.c_int, [_P, ctypes.c_longlong]),
    "rtproj_set_scaling": (ctypes.c_int, [_P, _P]),
    "rtproj_grad_workspace_bytes": (ctypes.c_size_t, [_P, _I64]),
    "rtproj_grad_A": (ctypes.c_int, [_P, _I64, _P, _I64, _P, _I64, _P, _I64, _P, _I64, _P, _I64, _P, ctypes.c_size_t]),
    "rtproj_sparse_workspace_bytes": (ctypes.c_size_t, [_I64, _I64, _I64, _I64, _I64, _I64, ctypes.POINTER(Opts)]),
    "rtproj_create_sparse": (ctypes.c_int, [ctypes.POINTER(_P), _I64, _I64, _I64, _P, _P, _P, _I64, _P, _P, _I64, _I64,
                                            _P, ctypes.c_size_t, _P, ctypes.POINTER(Opts)]),
}

PHASES = ["sketch", "qr", "gram", "factor", "apply_a", "apply_m", "apply_at", "slice"]


def library_path() -> str:
    return _build.LIB


def load_library():
    """Loads librtproj.so (built by ``_build.build()``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"librtproj.so is not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(code: int, where: str):
    if code != 0:
        raise RtprojError(code, where)


def default_opts() -> Opts:
    o = Opts()
    load_library().rtproj_default_opts(ctypes.byref(o))
    return o


def make_opts(mode="mixed", omega="gaussian", **slices) -> Opts:
    o = default_opts()
    o.mode = MODES[mode] if isinstance(mode, str) else int(mode)
    o.omega = OMEGAS[omega] if isinstance(omega, str) else int(omega)
    for k, v in slices.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def _dev_ptr(t: torch.Tensor) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


class Projector:
    """One matrix A bound to a workspace and a stream (see ``include/rtproj.h``)."""

    def __init__(self, A: torch.Tensor, l_max: int | None = None, k_max: int = 64, mode: str = "mixed",
                 omega: str = "gaussian", stream: torch.cuda.Stream | None = None, **slices):
        lib = load_library()
        if not (isinstance(A, torch.Tensor) and A.is_cuda and A.dtype in DTYPES and A.dim() == 2
                and A.stride(1) == 1 and A.stride(0) >= A.shape[1]):
            raise TypeError("A must be a CUDA float64 or float32 matrix with unit column stride")
        self.A = A
        self.dtype = A.dtype
        self.m, self.n = A.shape
        self.lda = A.stride(0)
        self.l_max = int(l_max if l_max is not None else min(self.n, 4 * self.m))
        self.k_max = int(k_max)
        self.device = A.device
        self.opts = make_opts(mode, omega, **slices)
        self.opts.dtype = DTYPES[A.dtype]
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._enter(A)   # create reads A on the handle's stream
        nbytes = lib.rtproj_workspace_bytes(self.m, self.n, self.l_max, self.k_max, ctypes.byref(self.opts))
        if nbytes == 0:
            raise RtprojError(1, "rtproj_workspace_bytes")
        # allocated on the handle's stream, so that the caching allocator reuses the memory
        # only after the work queued on that stream
        with torch.cuda.stream(self.stream):
            self.workspace = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            code = lib.rtproj_create(ctypes.byref(h), self.m, self.n, _dev_ptr(A), self.lda, self.l_max, self.k_max,
                                     _dev_ptr(self.workspace), ctypes.c_size_t(int(nbytes)),
                                     ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(self.opts))
        _check(code, "rtproj_create")
        self._h = h

    # -- lifecycle -------------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            load_library().rtproj_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- preconditioner ----------------------------------------------------------------
    def precondition(self, seed: int, l: int | None = None):
        l = self.l_max if l is None else int(l)
        self._enter()
        with torch.cuda.device(self.device):
            _check(load_library().rtproj_precondition(self._h, ctypes.c_uint64(seed), l), "rtproj_precondition")
        self.l = l
        return self

    def sketch(self, seed: int, l: int) -> torch.Tensor:
        cur = self._enter()
        with torch.cuda.stream(self.stream):
            S = torch.empty((self.m, l), dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            _check(load_library().rtproj_sketch(self._h, ctypes.c_uint64(seed), l, _dev_ptr(S), l), "rtproj_sketch")
        self._leave(cur, S)
        return S

    def export_state(self):
        import numpy as np
        R = np.empty((self.m, self.m))
        perm = np.empty(self.m, dtype=np.int32)
        L = np.empty((self.m, self.m))
        _check(load_library().rtproj_export_state(self._h, R.ctypes.data_as(_P), perm.ctypes.data_as(_P),
                                                  L.ctypes.data_as(_P)), "rtproj_export_state")
        return R, perm, L

    def info(self) -> dict:
        inf = Info()
        _check(load_library().rtproj_get_info(self._h, ctypes.byref(inf)), "rtproj_get_info")
        return {f: getattr(inf, f) for f, _ in Info._fields_}

    def timings(self) -> dict:
        """Per-phase device ms and counts since the last call (needs timing=1)."""
        import numpy as np
        ms = np.zeros(len(PHASES))
        cnt = np.zeros(len(PHASES), dtype=np.int64)
        _check(load_library().rtproj_get_timings(self._h, ms.ctypes.data_as(_P), cnt.ctypes.data_as(_P)),
               "rtproj_get_timings")
        return {p: (float(ms[i]), int(cnt[i])) for i, p in enumerate(PHASES)}

    def clear_status(self):
        _check(load_library().rtproj_clear_status(self._h), "rtproj_clear_status")

    def set_scaling(self, d: torch.Tensor | None):
        """The handle's matrix becomes A diag(d) (d: n float64 entries on the device; None
        restores A); the preconditioner is dropped. Needs scalable=1 at construction."""
        if d is not None and not (isinstance(d, torch.Tensor) and d.dtype == torch.float64 and d.device == self.device
                                  and d.dim() == 1 and d.shape[0] == self.n and d.stride(0) == 1):
            raise TypeError(f"d must be a contiguous float64 vector of {self.n} entries on {self.device}")
        cur = self._enter(*(() if d is None else (d,)))
        with torch.cuda.device(self.device):
            _check(load_library().rtproj_set_scaling(self._h, _dev_ptr(d) if d is not None else None),
                   "rtproj_set_scaling")
        self._leave(cur)

    def set_spin_limit(self, cycles: int):
        """Bound (SM clock cycles) on each grid-exchange wait of the QR and the Cholesky."""
        _check(load_library().rtproj_set_spin_limit(self._h, ctypes.c_longlong(int(cycles))), "rtproj_set_spin_limit")

    # -- apply -----------------------------------------------------------------------
    def _rhs(self, B: torch.Tensor) -> torch.Tensor:
        if not (isinstance(B, torch.Tensor) and B.dtype == self.dtype and B.device == self.device):
            raise TypeError(f"B must be a {self.dtype} tensor on {self.device}")
        if B.dim() == 1:
            B = B.reshape(1, -1)
        if B.dim() != 2 or B.shape[1] != self.n or B.stride(1) != 1 or B.stride(0) < self.n:
            raise TypeError(f"B must be k x {self.n} with unit column stride (one right-hand side per row)")
        if not (1 <= B.shape[0] <= self.k_max):
            raise TypeError(f"B has {B.shape[0]} rows; this handle takes 1..{self.k_max}")
        return B

    def _out(self, out: torch.Tensor, k: int, cols: int, name: str):
        if not (isinstance(out, torch.Tensor) and out.dtype == self.dtype and out.device == self.device
                and out.dim() == 2 and tuple(out.shape) == (k, cols) and out.stride(1) == 1 and out.stride(0) >= cols):
            raise TypeError(f"{name} must be a {k} x {cols} {self.dtype} tensor on {self.device} with unit column stride")
        return out

    def _enter(self, *inputs):
        """Orders the handle's stream after the caller's current stream (which produced the
        inputs) and keeps the inputs' memory from being reused before the handle's stream has
        read them."""
        cur = torch.cuda.current_stream(self.device)
        if cur != self.stream:
            self.stream.wait_stream(cur)
            for t in inputs:
                t.record_stream(self.stream)
        return cur

    def _leave(self, cur, *outputs):
        """Orders the caller's current stream after the handle's stream (which wrote the
        outputs), so the outputs can be read on either."""
        if cur != self.stream:
            cur.wait_stream(self.stream)
            for t in outputs:
                if t is not None:
                    t.record_stream(cur)

    def project(self, B: torch.Tensor, null: bool = True, row: bool = False, lstsq: bool = False,
                out_null: torch.Tensor | None = None):
        B = self._rhs(B)
        k = B.shape[0]
        if out_null is not None:
            self._out(out_null, k, self.n, "out_null")
        cur = self._enter(B)
        with torch.cuda.stream(self.stream):   # outputs belong to the handle's stream
            Z = (out_null if out_null is not None else torch.empty((k, self.n), dtype=self.dtype,
                                                                   device=self.device)) if null else None
            ROW = torch.empty((k, self.n), dtype=self.dtype, device=self.device) if row else None
            X = torch.empty((k, self.m), dtype=self.dtype, device=self.device) if lstsq else None
        ptr = lambda t: _dev_ptr(t) if t is not None else None
        ld = lambda t: t.stride(0) if t is not None else 0
        with torch.cuda.device(self.device):
            code = load_library().rtproj_project(self._h, _dev_ptr(B), B.stride(0), k, ptr(Z), ld(Z), ptr(ROW), ld(ROW),
                                                 ptr(X), ld(X))
        _check(code, "rtproj_project")
        self._leave(cur, Z, ROW, X)
        return Z, ROW, X

    def grad_A(self, H: torch.Tensor, Y: torch.Tensor, W: torch.Tensor, Zb: torch.Tensor) -> torch.Tensor:
        """dL/dA = -(H^* Y + W^* Zb) for L = sum_j <g_j, Z b_j> (rtproj_grad_A): H, W are
        lstsq(B), lstsq(G) (k x m); Y, Zb are Z G, Z B (k x n)."""
        k = H.shape[0]
        for t, cols, name in ((H, self.m, "H"), (W, self.m, "W"), (Y, self.n, "Y"), (Zb, self.n, "Zb")):
            self._out(t, k, cols, name)
        lib = load_library()
        nbytes = int(lib.rtproj_grad_workspace_bytes(self._h, k))
        if nbytes == 0:
            raise RtprojError(1, "rtproj_grad_workspace_bytes")
        cur = self._enter(H, Y, W, Zb)
        with torch.cuda.stream(self.stream):
            ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            dA = torch.empty((self.m, self.n), dtype=self.dtype, device=self.device)
        with torch.cuda.device(self.device):
            code = lib.rtproj_grad_A(self._h, k, _dev_ptr(H), H.stride(0), _dev_ptr(Y), Y.stride(0), _dev_ptr(W),
                                     W.stride(0), _dev_ptr(Zb), Zb.stride(0), _dev_ptr(dA), dA.stride(0),
                                     _dev_ptr(ws), ctypes.c_size_t(nbytes))
        _check(code, "rtproj_grad_A")
        self._leave(cur, dA)
        return dA

    def null_project(self, B, out=None):
        return self.project(B, null=True, out_null=out)[0]

    def row_project(self, B):
        return self.project(B, null=False, row=True)[1]

    def lstsq(self, B):
        return self.project(B, null=False, lstsq=True)[2]


class SparseProjector(Projector):
    """A = S + U V with S sparse (compressed sparse row, on the device) and an optional
    low-rank term U V (``rtproj_create_sparse``): the products with A cost O(nnz + r(m + n))
    and the apply's residuals are summed in double-double. The arrays are borrowed for the
    handle's lifetime (kept referenced here). The other methods are those of Projector;
    set_scaling is not supported."""

    def __init__(self, row_ptr: torch.Tensor, col_idx: torch.Tensor, val: torch.Tensor, n: int,
                 U: torch.Tensor | None = None, V: torch.Tensor | None = None, l_max: int | None = None,
                 k_max: int = 64, omega: str = "gaussian", stream: torch.cuda.Stream | None = None, **opts):
        lib = load_library()
        dev = val.device
        ok = (row_ptr.is_cuda and row_ptr.dtype == torch.int64 and row_ptr.dim() == 1 and row_ptr.is_contiguous()
              and col_idx.is_cuda and col_idx.dtype == torch.int32 and col_idx.dim() == 1 and col_idx.is_contiguous()
              and val.is_cuda and val.dtype == torch.float64 and val.dim() == 1 and val.is_contiguous()
              and row_ptr.device == dev and col_idx.device == dev and col_idx.numel() == val.numel())
        if not ok:
            raise TypeError("row_ptr (int64), col_idx (int32) and val (float64) must be contiguous CUDA vectors "
                            "on one device, col_idx and val of equal length")
        self.m, self.n = row_ptr.numel() - 1, int(n)
        r = 0
        if U is not None or V is not None:
            if U is None or V is None:
                raise TypeError("U and V go together")
            r = U.shape[1] if U.dim() == 2 else -1
            if not (U.is_cuda and U.dtype == torch.float64 and U.device == dev and U.is_contiguous()
                    and tuple(U.shape) == (self.m, r) and V.is_cuda and V.dtype == torch.float64
                    and V.device == dev and V.is_contiguous() and tuple(V.shape) == (r, self.n)):
                raise TypeError(f"U must be {self.m} x r and V r x {self.n}, contiguous float64 on {dev}")
        self._keep = (row_ptr, col_idx, val, U, V)
        self.A = None
        self.dtype = torch.float64
        self.lda = 0
        self.nnz, self.rank_lr = val.numel(), r
        self.l_max = int(l_max if l_max is not None else min(self.n, 4 * self.m))
        self.k_max = int(k_max)
        self.device = dev
        self.opts = make_opts("fp64", omega, **opts)
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self._enter(*[t for t in self._keep if t is not None])
        nbytes = lib.rtproj_sparse_workspace_bytes(self.m, self.n, self.nnz, r, self.l_max, self.k_max,
                                                   ctypes.byref(self.opts))
        if nbytes == 0:
            raise RtprojError(1, "rtproj_sparse_workspace_bytes")
        with torch.cuda.stream(self.stream):
            self.workspace = torch.empty(int(nbytes), dtype=torch.uint8, device=dev)
        h = ctypes.c_void_p()
        ptr = lambda t: _dev_ptr(t) if t is not None else None
        with torch.cuda.device(dev):
            code = lib.rtproj_create_sparse(ctypes.byref(h), self.m, self.n, self.nnz, _dev_ptr(row_ptr),
                                            _dev_ptr(col_idx), _dev_ptr(val), r, ptr(U), ptr(V), self.l_max,
                                            self.k_max, _dev_ptr(self.workspace), ctypes.c_size_t(int(nbytes)),
                                            ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(self.opts))
        _check(code, "rtproj_create_sparse")
        self._h = h

    def set_scaling(self, d):
        raise RtprojError(9, "set_scaling on a sparse handle")


def launch_count() -> int:
    """Kernels enqueued by librtproj since it was loaded."""
    return int(load_library().rtproj_launch_count())


def generate_omega(seed: int, n: int, l: int, omega: str = "gaussian", device="cuda") -> torch.Tensor:
    """The n x l test matrix G of Eq. 12 (float64), generated on the device as the sketch
    generates it (the sketch itself never stores G)."""
    dev = torch.device(device)
    G = torch.empty((n, l), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    with torch.cuda.device(dev):
        code = load_library().rtproj_generate_omega(ctypes.c_uint64(seed), n, l, OMEGAS[omega], _dev_ptr(G), l,
                                                    ctypes.c_void_p(stream.cuda_stream))
    _check(code, "rtproj_generate_omega")
    return G


def project_from_host(A_host: torch.Tensor, B_host: torch.Tensor, seed: int, l: int, device="cuda", **kw):
    """End-to-end call from host buffers: copies A and B to the device, preconditions,
    projects, and copies Z back (into pinned host memory)."""
    A = A_host.to(device, non_blocking=True)
    B = B_host.to(device, non_blocking=True)
    with Projector(A, l_max=l, k_max=B.shape[0], **kw) as P:
        P.precondition(seed, l)
        Z = P.null_project(B)
        out = torch.empty(Z.shape, dtype=Z.dtype, pin_memory=True)
        out.copy_(Z, non_blocking=True)
        torch.cuda.current_stream(A.device).synchronize()
    return out
