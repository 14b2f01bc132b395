"""Python binding of libsam (include/sam.h): argument marshalling only.

Every step of the SAM pipeline runs in the CUDA library; this module turns
torch tensors / numpy arrays into the plain pointers and sizes of the C ABI
and raises `SamError` on a non-zero status.  There is no CPU fallback: if
libsam.so is missing or no GPU is present, calls fail loudly.

Functions keep the C names (`sam_pattern_build`, `sam_build`,
`sam_build_batched`, `sam_residual`, `sam_apply`, `sam_build_backward`, ...)
as methods of `Handle`, which owns a `sam_handle` bound to a CUDA stream.
"""
from __future__ import annotations

import ctypes
import os
import threading
import weakref

import numpy as np

from . import build as _build

SAM_OK = 0
SAM_ERR_INVALID_ARG = 1
SAM_ERR_BAD_CSR = 2
SAM_ERR_RANK_DEFICIENT = 3
SAM_ERR_NONFINITE = 4
SAM_ERR_CUDA = 5
SAM_ERR_OOM = 6
SAM_ERR_TIMEOUT = 7
SAM_ERR_UNSUPPORTED = 8
SAM_FP64 = 0
SAM_FP32_REFINE = 1
SAM_FLAG_TRUSTED = 1
SAM_STATIC_MAX_ROWS = 1 << 19  # largest order sam_residual_static accepts
SAM_NUM_SIZE_CLASSES = 6
SAM_TAPE_OFF, SAM_TAPE_RECORD, SAM_TAPE_REPLAY = 0, 1, 2

PRECISIONS = {"fp64": SAM_FP64, "fp32r": SAM_FP32_REFINE}
SPARSIFY_MODES = {"global": 0, "tau": 1, "lfil": 2}
SAM_REFINE_AUTO = -1


def _steps(refine_steps) -> int:
    """refine_steps as an int; "auto" selects SAM_REFINE_AUTO."""
    return SAM_REFINE_AUTO if refine_steps == "auto" else int(refine_steps)

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_f64p = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p


class sam_csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int64), ("row_ptr", _vp), ("col_idx", _vp), ("val", _vp)]


class SamError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = int(status)
        super().__init__("%s failed: %s (status %d)" % (what, status_string(status), status))


_lib = None
_lock = threading.Lock()

# (name, restype, argtypes)
_SIGS = [
    ("sam_limits", None, [_i32p, _i32p]),
    ("sam_size_classes", ctypes.c_int32, [_i32p, _i32p, _i32p, _i32p, _i32p, ctypes.c_int]),
    ("sam_status_string", ctypes.c_char_p, [ctypes.c_int32]),
    ("sam_create", ctypes.c_int32, [ctypes.POINTER(_vp), _vp]),
    ("sam_destroy", ctypes.c_int32, [_vp]),
    ("sam_set_stream", ctypes.c_int32, [_vp, _vp]),
    ("sam_set_flags", ctypes.c_int32, [_vp, ctypes.c_uint32]),
    ("sam_sync", ctypes.c_int32, [_vp]),
    ("sam_pattern_build", ctypes.c_int32, [_vp, ctypes.POINTER(sam_csr), ctypes.c_int, ctypes.POINTER(_vp)]),
    ("sam_pattern_build_batched", ctypes.c_int32,
     [_vp, ctypes.c_int, ctypes.POINTER(sam_csr), ctypes.c_int, ctypes.POINTER(_vp)]),
    ("sam_pattern_from_csc", ctypes.c_int32, [_vp, ctypes.c_int32, ctypes.c_int64, _vp, _vp, ctypes.POINTER(_vp)]),
    ("sam_pattern_get", ctypes.c_int32, [_vp, _i32p, _i64p, ctypes.POINTER(_vp), ctypes.POINTER(_vp)]),
    ("sam_pattern_destroy", ctypes.c_int32, [_vp]),
    ("sam_build", ctypes.c_int32,
     [_vp, ctypes.POINTER(sam_csr), ctypes.POINTER(sam_csr), _vp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp,
      _vp]),
    ("sam_build_batched", ctypes.c_int32,
     [_vp, ctypes.c_int, ctypes.POINTER(sam_csr), ctypes.POINTER(sam_csr), ctypes.POINTER(_vp), ctypes.c_int,
      ctypes.c_int, _i64p, _vp, _vp, _vp, _vp, _vp, _f64p]),
    ("sam_residual", ctypes.c_int32,
     [_vp, ctypes.POINTER(sam_csr), ctypes.POINTER(sam_csr), ctypes.POINTER(sam_csr), _f64p, _f64p]),
    ("sam_apply", ctypes.c_int32, [_vp, ctypes.POINTER(sam_csr), _vp, _vp]),
    ("sam_apply_grad", ctypes.c_int32, [_vp, ctypes.POINTER(sam_csr), _vp, _vp, _vp]),
    ("sam_build_backward", ctypes.c_int32,
     [_vp, ctypes.POINTER(sam_csr), ctypes.POINTER(sam_csr), _vp, ctypes.c_int, ctypes.c_int, _vp, _vp,
      ctypes.c_double, _vp, _vp, _vp]),
    ("sam_tune", ctypes.c_int32,
     [_vp, ctypes.c_int, ctypes.POINTER(sam_csr), ctypes.POINTER(sam_csr), ctypes.POINTER(_vp), ctypes.c_int,
      ctypes.c_int, ctypes.c_char_p]),
    ("sam_build_multi", ctypes.c_int32,
     [_vp, ctypes.c_int, ctypes.POINTER(sam_csr), ctypes.POINTER(sam_csr), ctypes.POINTER(_vp), ctypes.c_int,
      ctypes.c_int, _i64p, _vp, _vp, _vp, _vp, _vp, _f64p]),
    ("sam_build_backward_batched", ctypes.c_int32,
     [_vp, ctypes.c_int, ctypes.POINTER(sam_csr), ctypes.POINTER(sam_csr), ctypes.POINTER(_vp), ctypes.c_int,
      ctypes.c_int, _i64p, _vp, _vp, ctypes.c_double, _vp, _vp, _vp]),
    ("sam_plan_create", ctypes.c_int32,
     [_vp, ctypes.c_int, ctypes.POINTER(sam_csr), ctypes.POINTER(sam_csr), ctypes.c_int, ctypes.POINTER(_vp),
      ctypes.c_int, ctypes.c_int, _i64p, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(_vp)]),
    ("sam_plan_execute", ctypes.c_int32, [_vp]),
    ("sam_plan_launches", ctypes.c_int32, [_vp, _i64p]),
    ("sam_plan_destroy", ctypes.c_int32, [_vp]),
    ("sam_refine_stats", ctypes.c_int32, [_vp, _i64p, ctypes.c_int]),
    ("sam_sparsify", ctypes.c_int32,
     [_vp, ctypes.POINTER(sam_csr), ctypes.c_int, ctypes.c_double, _vp, _vp, _vp, _i64p]),
    ("sam_sparsify_batched", ctypes.c_int32,
     [_vp, ctypes.c_int, ctypes.POINTER(sam_csr), ctypes.c_int, ctypes.c_double, _vp, _vp, _vp, _i64p]),
    ("sam_set_tile_variants", ctypes.c_int32, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
    ("sam_get_tile_variants", ctypes.c_int32, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
    ("sam_set_bin_schedule", ctypes.c_int32, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
    ("sam_get_bin_schedule", ctypes.c_int32, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
    ("sam_factor_tape_bytes", ctypes.c_int32, [_vp, ctypes.c_int, ctypes.POINTER(_vp), ctypes.c_int, _i64p]),
    ("sam_set_factor_tape", ctypes.c_int32, [_vp, ctypes.c_int, _vp, ctypes.c_int64]),
    ("sam_profile", ctypes.c_int32, [_vp, ctypes.c_int]),
    ("sam_profile_read", ctypes.c_int32, [_vp, _i64p, ctypes.POINTER(ctypes.c_double), _i64p]),
    ("sam_peak_flops", ctypes.c_int32, [_vp, ctypes.c_double, _f64p, _f64p]),
    ("sam_gmres", ctypes.c_int32,
     [_vp, ctypes.POINTER(sam_csr), ctypes.POINTER(sam_csr), ctypes.POINTER(sam_csr), _vp, _vp, ctypes.c_int,
      ctypes.c_int, ctypes.c_double, _i32p, _f64p, _vp]),
    ("sam_gmres_batched", ctypes.c_int32,
     [_vp, ctypes.c_int, ctypes.POINTER(sam_csr), ctypes.POINTER(sam_csr), ctypes.POINTER(sam_csr), _vp, _vp,
      ctypes.c_int, ctypes.c_int, ctypes.c_double, _i32p, _f64p, _vp]),
    ("sam_residual_static", ctypes.c_int32,
     [_vp, ctypes.POINTER(sam_csr), ctypes.POINTER(sam_csr), ctypes.POINTER(sam_csr), _vp, _vp]),
]


def lib_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = False):
    """Load libsam.so (building it first if asked and it is missing)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB_PATH
            if not os.path.exists(path):
                if not build_if_missing:
                    raise RuntimeError("libsam.so is not built (%s); run paper_2406_17656_gb300.build.build()" % path)
                _build.build()
            lib = ctypes.CDLL(path)
            for name, res, args in _SIGS:
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def exported_symbols() -> list[str]:
    return [s[0] for s in _SIGS]


def status_string(s: int) -> str:
    try:
        return load().sam_status_string(int(s)).decode()
    except Exception:  # library not loadable: still give a message
        return "status %d" % s


def limits() -> tuple[int, int]:
    r, c = ctypes.c_int32(), ctypes.c_int32()
    load().sam_limits(ctypes.byref(r), ctypes.byref(c))
    return r.value, c.value


def size_classes() -> dict:
    """The size classes of the column problems (include/sam.h): per class
    the largest |I_j|, |J_j|, nnz(B_j), |I_j| (|J_j| + 1) and the number of
    tile variants."""
    C = SAM_NUM_SIZE_CLASSES
    r, c, e, t, v = [(ctypes.c_int32 * C)() for _ in range(5)]
    _check(load().sam_size_classes(r, c, e, t, v, C), "sam_size_classes")
    return {"max_rows": list(r), "max_cols": list(c), "max_entries": list(e), "max_tile": list(t),
            "variants": list(v)}


def _check(st: int, what: str):
    if st != SAM_OK:
        raise SamError(st, what)


def _addr(x) -> int:
    """Raw address of a torch tensor or numpy array (contiguity required)."""
    if x is None:
        return 0
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return int(x.data_ptr())
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be contiguous")
        return int(x.ctypes.data)
    raise TypeError("expected a torch tensor or numpy array, got %r" % type(x))


def sam_residual_static(A_k: "Csr", M_k: "Csr", A_0: "Csr", out, status=None, stream=None):
    """||A_k M_k - A_0||_F and its ratio to ||A_0||_F into the device array
    `out` (2 float64) without allocating device memory (see include/sam.h);
    all arrays must be on the device.  Asynchronous on `stream` (default:
    torch's current stream)."""
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    a, m, z = A_k.c(), M_k.c(), A_0.c()
    _check(load().sam_residual_static(_vp(int(stream.cuda_stream)), ctypes.byref(a), ctypes.byref(m), ctypes.byref(z),
                                      _addr(out), _addr(status)), "sam_residual_static")
    return out


class Csr:
    """A CSR matrix given by three arrays (torch tensors on any device, or
    numpy arrays): indptr int32[n+1], indices int32[nnz], data float64[nnz]."""

    def __init__(self, indptr, indices, data=None, n: int | None = None):
        self.indptr, self.indices, self.data = indptr, indices, data
        self.n = int(n if n is not None else len(indptr) - 1)
        self.nnz = int(indices.shape[0])
        for a, dt in ((indptr, "int32"), (indices, "int32")):
            if str(a.dtype).split(".")[-1] != dt:
                raise TypeError("CSR index arrays must be int32")
        if data is not None and str(data.dtype).split(".")[-1] != "float64":
            raise TypeError("CSR values must be float64")

    def c(self) -> sam_csr:
        return sam_csr(self.n, self.nnz, _addr(self.indptr), _addr(self.indices), _addr(self.data))

    @staticmethod
    def from_host(m, device="cuda") -> "Csr":
        """Copy an object with n/indptr/indices/data numpy arrays to torch tensors on `device`."""
        import torch

        return Csr(torch.from_numpy(np.ascontiguousarray(m.indptr, np.int32)).to(device),
                   torch.from_numpy(np.ascontiguousarray(m.indices, np.int32)).to(device),
                   torch.from_numpy(np.ascontiguousarray(m.data, np.float64)).to(device), n=m.n)


class _CudaView:
    """Exposes a library-owned device array through __cuda_array_interface__."""

    def __init__(self, ptr: int, count: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (count,), "typestr": typestr, "data": (ptr, False), "version": 3}


class Pattern:
    """A map sparsity pattern owned by libsam (CSC: colptr[n+1], rowidx[nnz])."""

    def __init__(self, handle: "Handle", ptr: int):
        self.handle, self.ptr = handle, ptr
        handle._patterns.add(self)
        n, nnz = ctypes.c_int32(), ctypes.c_int64()
        _check(load().sam_pattern_get(ptr, ctypes.byref(n), ctypes.byref(nnz), None, None), "sam_pattern_get")
        self.n, self.nnz = n.value, nnz.value
        self._cp = self._ri = None

    def _views(self):
        if self._cp is None:
            cp, ri = _vp(), _vp()
            _check(load().sam_pattern_get(self.ptr, None, None, ctypes.byref(cp), ctypes.byref(ri)),
                   "sam_pattern_get")
            self._cp, self._ri = cp.value, ri.value
        return self._cp, self._ri

    def colptr(self):
        import torch

        return torch.as_tensor(_CudaView(self._views()[0], self.n + 1, "<i4"), device="cuda")

    def rowidx(self):
        import torch

        return torch.as_tensor(_CudaView(self._views()[1], self.nnz, "<i4"), device="cuda")

    def destroy(self):
        # a pattern lives in its handle's memory pool: once the handle is
        # closed the pool has released it, and the pattern must not be touched
        if self.ptr and getattr(self.handle, "ptr", 0):
            load().sam_pattern_destroy(self.ptr)
        self.ptr = 0

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class Plan:
    """A captured numeric rebuild (sam_plan_create): `execute()` replays the
    whole value-dependent build as one CUDA graph.  Keeps the arrays it was
    made from alive."""

    def __init__(self, handle: "Handle", ptr: int, keep: tuple, offsets, outputs):
        self.handle, self.ptr, self._keep = handle, ptr, keep
        self.offsets = offsets
        self.M_row_ptr, self.M_col_idx, self.M_val, self.col_status, self.res2, self.fro2 = outputs
        handle._patterns.add(self)

    def execute(self):
        _check(load().sam_plan_execute(self.ptr), "sam_plan_execute")

    def launches(self) -> int:
        n = ctypes.c_int64()
        _check(load().sam_plan_launches(self.ptr, ctypes.byref(n)), "sam_plan_launches")
        return n.value

    def destroy(self):
        if self.ptr and getattr(self.handle, "ptr", 0):
            load().sam_plan_destroy(self.ptr)
        self.ptr = 0

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class Handle:
    """A sam_handle bound to a CUDA stream (default: torch's current stream)."""

    def __init__(self, stream=None, trusted: bool = False):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("libsam needs a CUDA GPU")
        lib = load()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self._patterns = weakref.WeakSet()
        h = _vp()
        _check(lib.sam_create(ctypes.byref(h), _vp(int(stream.cuda_stream))), "sam_create")
        self.ptr = h.value
        if trusted:
            _check(lib.sam_set_flags(self.ptr, SAM_FLAG_TRUSTED), "sam_set_flags")

    def close(self):
        if getattr(self, "ptr", 0):
            for p in list(getattr(self, "_patterns", ())):
                p.destroy()
            load().sam_destroy(self.ptr)
            self.ptr = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sam_sync(self):
        _check(load().sam_sync(self.ptr), "sam_sync")

    def sam_set_flags(self, flags: int):
        _check(load().sam_set_flags(self.ptr, int(flags)), "sam_set_flags")

    # -------------------------------------------------------------- patterns
    def sam_pattern_build(self, A: Csr, level: int) -> Pattern:
        out = _vp()
        c = A.c()
        _check(load().sam_pattern_build(self.ptr, ctypes.byref(c), int(level), ctypes.byref(out)), "sam_pattern_build")
        return Pattern(self, out.value)

    def sam_pattern_build_batched(self, As: list, level: int) -> list:
        K = len(As)
        arr = (sam_csr * K)(*[a.c() for a in As])
        outs = (_vp * K)()
        _check(load().sam_pattern_build_batched(self.ptr, K, arr, int(level), outs), "sam_pattern_build_batched")
        return [Pattern(self, outs[k]) for k in range(K)]

    def sam_pattern_from_csc(self, n: int, colptr, rowidx) -> Pattern:
        out = _vp()
        _check(load().sam_pattern_from_csc(self.ptr, int(n), int(rowidx.shape[0]), _addr(colptr), _addr(rowidx),
                                           ctypes.byref(out)), "sam_pattern_from_csc")
        return Pattern(self, out.value)

    # ----------------------------------------------------------------- build
    def sam_build(self, A_k: Csr, A_0: Csr, S: Pattern, precision="fp32r", refine_steps: int = 1,
                  out=None, col_status=None, res2=None):
        """Build the map on pattern S; `out` = (indptr, indices, data) arrays
        (allocated on the device if None).  Returns `out`."""
        import torch

        prec = PRECISIONS.get(precision, precision)
        if out is None:
            dev = A_k.indptr.device if hasattr(A_k.indptr, "device") else "cuda"
            out = (torch.empty(A_k.n + 1, dtype=torch.int32, device=dev),
                   torch.empty(S.nnz, dtype=torch.int32, device=dev),
                   torch.empty(S.nnz, dtype=torch.float64, device=dev))
        a, z = A_k.c(), A_0.c()
        _check(load().sam_build(self.ptr, ctypes.byref(a), ctypes.byref(z), S.ptr, int(prec), _steps(refine_steps),
                                _addr(out[0]), _addr(out[1]), _addr(out[2]), _addr(col_status), _addr(res2)),
               "sam_build")
        return out

    def sam_build_batched(self, A_ks: list, A_0, Ss: list, precision="fp32r", refine_steps: int = 1,
                          M_row_ptr=None, M_col_idx=None, M_val=None, col_status=None, res2=None,
                          want_fro: bool = False, offsets=None):
        """K maps in one pass.  A_0 is the shared target (sam_build_batched)
        or a list of K targets, one per map (sam_build_multi).  Output arrays
        are allocated on the device when None.  Returns (offsets,
        M_row_ptr[K*(n+1)], M_col_idx, M_val, fro)."""
        import torch

        K = len(A_ks)
        prec = PRECISIONS.get(precision, precision)
        multi = isinstance(A_0, (list, tuple))
        if multi and len(A_0) != K:
            raise ValueError("one target per map")
        n = (A_0[0] if multi else A_0).n
        if offsets is None:
            offsets = np.zeros(K + 1, dtype=np.int64)
            offsets[1:] = np.cumsum([s.nnz for s in Ss])
        tot = int(offsets[-1])
        if M_row_ptr is None:
            M_row_ptr = torch.empty(K * (n + 1), dtype=torch.int32, device="cuda")
        if M_col_idx is None:
            M_col_idx = torch.empty(tot, dtype=torch.int32, device="cuda")
        if M_val is None:
            M_val = torch.empty(tot, dtype=torch.float64, device="cuda")
        arr = (sam_csr * K)(*[a.c() for a in A_ks])
        if multi:
            z = (sam_csr * K)(*[a.c() for a in A_0])
            zp, fn, name = z, load().sam_build_multi, "sam_build_multi"
        else:
            z = A_0.c()
            zp, fn, name = ctypes.byref(z), load().sam_build_batched, "sam_build_batched"
        pats = (_vp * K)(*[s.ptr for s in Ss])
        fro = np.zeros(K, dtype=np.float64) if want_fro else None
        _check(fn(self.ptr, K, arr, zp, pats, int(prec), _steps(refine_steps), offsets.ctypes.data_as(_i64p),
                  _addr(M_row_ptr), _addr(M_col_idx), _addr(M_val), _addr(col_status), _addr(res2),
                  fro.ctypes.data_as(_f64p) if fro is not None else None), name)
        return offsets, M_row_ptr, M_col_idx, M_val, fro

    # ----------------------------------------------------------- sparsify
    def sam_sparsify(self, A: Csr, mode: str, param: float) -> Csr:
        """Sparsified A~ of Sec. 4 (mode "global", "tau" or "lfil"), as a
        device Csr holding only the kept entries."""
        import torch

        rp = torch.empty(A.n + 1, dtype=torch.int32, device="cuda")
        ci = torch.empty(max(A.nnz, 1), dtype=torch.int32, device="cuda")
        v = torch.empty(max(A.nnz, 1), dtype=torch.float64, device="cuda")
        nnz = ctypes.c_int64()
        a = A.c()
        _check(load().sam_sparsify(self.ptr, ctypes.byref(a), SPARSIFY_MODES[mode], float(param), _addr(rp),
                                   _addr(ci), _addr(v), ctypes.byref(nnz)), "sam_sparsify")
        k = int(nnz.value)
        return Csr(rp, ci[:k], v[:k], n=A.n)

    def sam_sparsify_batched(self, As: list, mode: str, param: float) -> list:
        """sam_sparsify of K matrices of one order in a single pass; returns
        K device Csr views of the kept entries."""
        import torch

        K = len(As)
        n = As[0].n
        tot = sum(a.nnz for a in As)
        rp = torch.empty(K * (n + 1), dtype=torch.int32, device="cuda")
        ci = torch.empty(max(tot, 1), dtype=torch.int32, device="cuda")
        v = torch.empty(max(tot, 1), dtype=torch.float64, device="cuda")
        off = np.zeros(K + 1, dtype=np.int64)
        arr = (sam_csr * K)(*[a.c() for a in As])
        _check(load().sam_sparsify_batched(self.ptr, K, arr, SPARSIFY_MODES[mode], float(param), _addr(rp), _addr(ci),
                                           _addr(v), off.ctypes.data_as(_i64p)), "sam_sparsify_batched")
        return [Csr(rp[k * (n + 1):(k + 1) * (n + 1)], ci[off[k]:off[k + 1]], v[off[k]:off[k + 1]], n=n)
                for k in range(K)]

    # -------------------------------------------------------------- residual
    def sam_residual(self, A_k: Csr, M_k: Csr, A_0: Csr):
        fro, rel = ctypes.c_double(), ctypes.c_double()
        a, m, z = A_k.c(), M_k.c(), A_0.c()
        _check(load().sam_residual(self.ptr, ctypes.byref(a), ctypes.byref(m), ctypes.byref(z), ctypes.byref(fro),
                                   ctypes.byref(rel)), "sam_residual")
        return fro.value, rel.value

    def sam_apply(self, M_k: Csr, x, y=None):
        import torch

        if y is None:
            y = torch.empty_like(x) if hasattr(x, "data_ptr") else np.empty_like(x)
        m = M_k.c()
        _check(load().sam_apply(self.ptr, ctypes.byref(m), _addr(x), _addr(y)), "sam_apply")
        return y

    def sam_apply_grad(self, M_k: Csr, x, dy, dM_val=None):
        """dL/dM values of y = M_k x given dy = dL/dy: dM_val[e] = dy[i] x[c]."""
        import torch

        if dM_val is None:
            dM_val = torch.empty(M_k.nnz, dtype=torch.float64, device=x.device) if hasattr(x, "data_ptr") else \
                np.empty(M_k.nnz, dtype=np.float64)
        m = M_k.c()
        _check(load().sam_apply_grad(self.ptr, ctypes.byref(m), _addr(x), _addr(dy), _addr(dM_val)),
               "sam_apply_grad")
        return dM_val

    def sam_gmres(self, A: Csr, b, x=None, M: Csr | None = None, P_0: Csr | None = None, restart: int = 30,
                  maxiter: int = 1000, rtol: float = 1e-8, history=None):
        """Restarted GMRES for A x = b with the right preconditioner
        z = M (P_0 v) (either operator may be None = identity).  x holds the
        initial guess (zeros if None) and receives the solution.  history
        (nullable, float64[maxiter], device or host) gets the residual
        estimate / ||b|| after every step.  Returns (x, iterations, relres)."""
        import torch

        if x is None:
            x = torch.zeros_like(b) if hasattr(b, "data_ptr") else np.zeros_like(b)
        its, rel = ctypes.c_int32(), ctypes.c_double()
        a = A.c()
        m = M.c() if M is not None else None
        p = P_0.c() if P_0 is not None else None
        _check(load().sam_gmres(self.ptr, ctypes.byref(a), ctypes.byref(m) if m is not None else None,
                                ctypes.byref(p) if p is not None else None, _addr(b), _addr(x), int(restart),
                                int(maxiter), float(rtol), ctypes.byref(its), ctypes.byref(rel), _addr(history)),
               "sam_gmres")
        return x, its.value, rel.value

    def sam_gmres_batched(self, As: list, b, x=None, Ms: list | None = None, P_0: Csr | None = None,
                          restart: int = 30, maxiter: int = 1000, rtol: float = 1e-8, history=None):
        """K independent restarted GMRES solves A_k x_k = b_k with the right
        preconditioners M_k (P_0 v), in the same launches.  b, x: [K*n]
        (system k at k*n).  Returns (x, iterations[K], relres[K])."""
        import torch

        K = len(As)
        if x is None:
            x = torch.zeros_like(b) if hasattr(b, "data_ptr") else np.zeros_like(b)
        its = np.zeros(K, dtype=np.int32)
        rel = np.zeros(K, dtype=np.float64)
        a = (sam_csr * K)(*[m.c() for m in As])
        m = (sam_csr * K)(*[q.c() for q in Ms]) if Ms is not None else None
        p = P_0.c() if P_0 is not None else None
        _check(load().sam_gmres_batched(self.ptr, K, a, m, ctypes.byref(p) if p is not None else None, _addr(b),
                                        _addr(x), int(restart), int(maxiter), float(rtol),
                                        its.ctypes.data_as(_i32p), rel.ctypes.data_as(_f64p), _addr(history)),
               "sam_gmres_batched")
        return x, its, rel

    def sam_build_backward(self, A_k: Csr, A_0: Csr, S: Pattern, M_val, dM_val=None, precision="fp32r",
                           refine_steps: int = 1, resid_weight: float = 0.0, dA_k_val=None, dA_0_val=None,
                           dM_resid=None):
        """Gradients of <dM, M> + resid_weight ||A_k M - A_0||_F^2 with respect
        to the values of A_k and A_0 (CSR orders); see include/sam.h."""
        import torch

        prec = PRECISIONS.get(precision, precision)
        if dA_k_val is None:
            dA_k_val = torch.empty(A_k.nnz, dtype=torch.float64, device="cuda")
        if dA_0_val is None:
            dA_0_val = torch.empty(A_0.nnz, dtype=torch.float64, device="cuda")
        a, z = A_k.c(), A_0.c()
        _check(load().sam_build_backward(self.ptr, ctypes.byref(a), ctypes.byref(z), S.ptr, int(prec),
                                         _steps(refine_steps), _addr(M_val), _addr(dM_val), float(resid_weight),
                                         _addr(dA_k_val), _addr(dA_0_val), _addr(dM_resid)), "sam_build_backward")
        return dA_k_val, dA_0_val

    def sam_build_backward_batched(self, A_ks: list, A_0s: list, Ss: list, M_val, dM_val=None, precision="fp32r",
                                   refine_steps: int = 1, resid_weight: float = 0.0, offsets=None, dA_k_val=None,
                                   dA_0_val=None, dM_resid=None):
        """K maps, map k against its own target A_0s[k]; values concatenated
        in map order (see include/sam.h).  Returns (dA_k_val, dA_0_val)."""
        import torch

        K = len(A_ks)
        prec = PRECISIONS.get(precision, precision)
        if offsets is None:
            offsets = np.zeros(K + 1, dtype=np.int64)
            offsets[1:] = np.cumsum([s.nnz for s in Ss])
        if dA_k_val is None:
            dA_k_val = torch.empty(sum(a.nnz for a in A_ks), dtype=torch.float64, device="cuda")
        if dA_0_val is None:
            dA_0_val = torch.empty(sum(a.nnz for a in A_0s), dtype=torch.float64, device="cuda")
        arr = (sam_csr * K)(*[a.c() for a in A_ks])
        z = (sam_csr * K)(*[a.c() for a in A_0s])
        pats = (_vp * K)(*[s.ptr for s in Ss])
        _check(load().sam_build_backward_batched(self.ptr, K, arr, z, pats, int(prec), _steps(refine_steps),
                                                 offsets.ctypes.data_as(_i64p), _addr(M_val), _addr(dM_val),
                                                 float(resid_weight), _addr(dA_k_val), _addr(dA_0_val),
                                                 _addr(dM_resid)), "sam_build_backward_batched")
        return dA_k_val, dA_0_val

    # ------------------------------------------------------------------ plans
    def sam_plan_create(self, A_ks: list, A_0, Ss: list, precision="fp32r", refine_steps: int = 1,
                        want_status: bool = False, want_res2: bool = False, want_fro2: bool = True) -> Plan:
        """Capture the batched build of these device matrices (A_0 shared, or
        a list of one target per map) as a replayable plan; outputs are
        allocated here and live on the returned Plan."""
        import torch

        K = len(A_ks)
        prec = PRECISIONS.get(precision, precision)
        multi = isinstance(A_0, (list, tuple))
        tg = list(A_0) if multi else [A_0]
        n = tg[0].n
        offsets = np.zeros(K + 1, dtype=np.int64)
        offsets[1:] = np.cumsum([s.nnz for s in Ss])
        tot = int(offsets[-1])
        dev = "cuda"
        rp = torch.empty(K * (n + 1), dtype=torch.int32, device=dev)
        ci = torch.empty(tot, dtype=torch.int32, device=dev)
        v = torch.empty(tot, dtype=torch.float64, device=dev)
        st = torch.empty(K * n, dtype=torch.int32, device=dev) if want_status else None
        r2 = torch.empty(K * n, dtype=torch.float64, device=dev) if want_res2 else None
        f2 = torch.empty(K, dtype=torch.float64, device=dev) if want_fro2 else None
        arr = (sam_csr * K)(*[a.c() for a in A_ks])
        z = (sam_csr * len(tg))(*[a.c() for a in tg])
        pats = (_vp * K)(*[s.ptr for s in Ss])
        out = _vp()
        _check(load().sam_plan_create(self.ptr, K, arr, z, len(tg), pats, int(prec), _steps(refine_steps),
                                      offsets.ctypes.data_as(_i64p), _addr(rp), _addr(ci), _addr(v), _addr(st),
                                      _addr(r2), _addr(f2), ctypes.byref(out)), "sam_plan_create")
        return Plan(self, out.value, (tuple(A_ks), tuple(tg)), offsets, (rp, ci, v, st, r2, f2))

    # ---------------------------------------------------------------- tuning
    def sam_tune(self, A_ks: list, A_0: Csr, Ss: list, precision="fp32r", refine_steps: int = 1,
                 cache_path: str | None = None):
        """Choose the tile variant of every size class and the bin schedule
        on these problems (kept in the handle); returns the chosen variants
        (the schedule: sam_get_bin_schedule)."""
        K = len(A_ks)
        prec = PRECISIONS.get(precision, precision)
        arr = (sam_csr * K)(*[a.c() for a in A_ks])
        z = A_0.c()
        pats = (_vp * K)(*[s.ptr for s in Ss])
        _check(load().sam_tune(self.ptr, K, arr, ctypes.byref(z), pats, int(prec), _steps(refine_steps),
                               cache_path.encode() if cache_path else None), "sam_tune")
        return self.sam_get_tile_variants()

    def sam_set_tile_variants(self, variants):
        v = (ctypes.c_int * SAM_NUM_SIZE_CLASSES)(*[int(x) for x in variants])
        _check(load().sam_set_tile_variants(self.ptr, v, len(variants)), "sam_set_tile_variants")

    def sam_set_bin_schedule(self, to):
        v = (ctypes.c_int * SAM_NUM_SIZE_CLASSES)(*[int(x) for x in to])
        _check(load().sam_set_bin_schedule(self.ptr, v, len(to)), "sam_set_bin_schedule")

    def sam_get_bin_schedule(self):
        """The size class that solves each natural size class's columns."""
        v = (ctypes.c_int * SAM_NUM_SIZE_CLASSES)()
        _check(load().sam_get_bin_schedule(self.ptr, v, SAM_NUM_SIZE_CLASSES), "sam_get_bin_schedule")
        return list(v)

    def sam_factor_tape_bytes(self, Ss: list, precision="fp32r") -> int:
        """Bytes of the factor tape of the maps on patterns Ss."""
        pats = (_vp * len(Ss))(*[s.ptr for s in Ss])
        out = ctypes.c_int64(0)
        _check(load().sam_factor_tape_bytes(self.ptr, len(Ss), pats, int(PRECISIONS.get(precision, precision)),
                                            ctypes.byref(out)), "sam_factor_tape_bytes")
        return int(out.value)

    def sam_set_factor_tape(self, mode: int, buf=None):
        """SAM_TAPE_RECORD / SAM_TAPE_REPLAY with a device buffer (a tensor
        of at least sam_factor_tape_bytes bytes), or SAM_TAPE_OFF."""
        if mode == SAM_TAPE_OFF or buf is None:
            _check(load().sam_set_factor_tape(self.ptr, int(mode), None, 0), "sam_set_factor_tape")
            return
        nbytes = buf.numel() * buf.element_size()
        _check(load().sam_set_factor_tape(self.ptr, int(mode), ctypes.c_void_p(buf.data_ptr()), nbytes),
               "sam_set_factor_tape")

    def sam_refine_stats(self):
        """[one step, two steps, FP64 re-solve] column counts of the last
        build with refine_steps="auto"."""
        c = (ctypes.c_int64 * 3)()
        _check(load().sam_refine_stats(self.ptr, c, 3), "sam_refine_stats")
        return list(c)

    def sam_get_tile_variants(self):
        v = (ctypes.c_int * SAM_NUM_SIZE_CLASSES)()
        _check(load().sam_get_tile_variants(self.ptr, v, SAM_NUM_SIZE_CLASSES), "sam_get_tile_variants")
        return list(v)

    def sam_profile(self, enable: bool):
        _check(load().sam_profile(self.ptr, int(bool(enable))), "sam_profile")

    def sam_profile_read(self):
        """(kernel launches, per-size-class least-squares ms, per-class launches)."""
        n = ctypes.c_int64()
        ms = (ctypes.c_double * SAM_NUM_SIZE_CLASSES)()
        cnt = (ctypes.c_int64 * SAM_NUM_SIZE_CLASSES)()
        _check(load().sam_profile_read(self.ptr, ctypes.byref(n), ms, cnt), "sam_profile_read")
        return n.value, list(ms), list(cnt)

    def sam_peak_flops(self, ms: float = 50.0):
        f32, f64 = ctypes.c_double(), ctypes.c_double()
        _check(load().sam_peak_flops(self.ptr, float(ms), ctypes.byref(f32), ctypes.byref(f64)), "sam_peak_flops")
        return f32.value, f64.value
