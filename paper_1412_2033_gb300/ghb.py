"""Python binding of the ghb C ABI (include/ghb.h): argument marshalling only.

Every step of the method runs in the CUDA library ``lib/libghb.so``; this module
loads it with ctypes, converts arguments, and uses PyTorch only for device
memory and streams.  There is no CPU fallback: if the library is missing or
cannot be loaded, importing the functions raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from .build import LIB

GHB_OK, GHB_ERR_INVALID, GHB_ERR_OOM, GHB_ERR_NOT_CONVERGED, GHB_ERR_BREAKDOWN, GHB_ERR_CUDA = range(6)
GHB_BOX, GHB_DISK, GHB_SPHERE = 0, 1, 2
GHB_PRIMAL, GHB_DUAL, GHB_GANI_PRIMAL, GHB_GANI_DUAL = 0, 1, 2, 3
GHB_FP64, GHB_MIXED, GHB_FP32 = 0, 1, 2
GHB_FORM_DOUBLE_GRID, GHB_FORM_REDUCED = 0, 1

STATUS_NAMES = {0: "GHB_OK", 1: "GHB_ERR_INVALID", 2: "GHB_ERR_OOM", 3: "GHB_ERR_NOT_CONVERGED",
                4: "GHB_ERR_BREAKDOWN", 5: "GHB_ERR_CUDA"}

# every symbol include/ghb.h declares
EXPORTS = ["ghb_default_options", "ghb_create", "ghb_set_coeffs", "ghb_set_options", "ghb_set_stream",
           "ghb_get_grid", "ghb_field_elems", "ghb_matvec", "ghb_solve_primal", "ghb_solve_dual",
           "ghb_gram", "ghb_bounds", "ghb_table_elems", "ghb_grid_elems", "ghb_copy_table",
           "ghb_copy_grid_values", "ghb_device_bytes", "ghb_last_error", "ghb_destroy", "ghb_version",
           "ghb_profile", "ghb_profile_read", "ghb_batch_create", "ghb_batch_submit", "ghb_batch_step",
           "ghb_batch_run", "ghb_batch_results", "ghb_batch_stats", "ghb_batch_destroy", "ghb_gram_noalloc",
           "ghb_tune_get", "ghb_tune_set", "ghb_tune_reset", "ghb_bounds_gani", "ghb_solve_ex", "ghb_prolong",
           "ghb_create_image", "ghb_set_image", "ghb_set_form"]

PROFILE_CLASSES = ["coeff", "col1_inv_pupdate", "col1_inv", "col2_inv", "row_matvec", "col2_fwd", "col1_fwd",
                   "project_dot", "update", "project", "residual", "gram_row", "misc"]


class GhbPhase(ctypes.Structure):
    _fields_ = [("shape", ctypes.c_int32), ("pad_", ctypes.c_int32), ("center", ctypes.c_double * 3),
                ("size", ctypes.c_double * 3), ("value", ctypes.c_double)]


class GhbOptions(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("inner_tol", ctypes.c_double), ("max_outer", ctypes.c_int32), ("M", ctypes.c_int32 * 3)]


class GhbSolveInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("outer_iters", ctypes.c_int32),
                ("matvecs_fp64", ctypes.c_int32), ("matvecs_fp32", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("relres", ctypes.c_double), ("energy", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad_"}


class GhbResult(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("d", ctypes.c_int32), ("status", ctypes.c_int32),
                ("upper", ctypes.c_double * 9), ("lower", ctypes.c_double * 9), ("info", GhbSolveInfo * 6),
                ("seconds_queued", ctypes.c_double), ("seconds_total", ctypes.c_double)]

    def as_dict(self):
        d = self.d
        return {"id": self.id, "d": d, "status": self.status,
                "upper": np.array(self.upper[: d * d]).reshape(d, d),
                "lower": np.array(self.lower[: d * d]).reshape(d, d),
                "infos": [self.info[i].as_dict() for i in range(2 * d)],
                "seconds_queued": self.seconds_queued, "seconds_total": self.seconds_total}


class GhbError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load_library(path: str = LIB) -> ctypes.CDLL:
    """Load lib/libghb.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"ghb CUDA library not built: {path} is missing "
                          "(run paper_1412_2033_gb300.build.build())")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i32, i64, dbl = ctypes.c_int, ctypes.c_int64, ctypes.c_double
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    sig = {
        "ghb_default_options": (None, [ctypes.POINTER(GhbOptions)]),
        "ghb_create": (i32, [ctypes.POINTER(P), i32, ip, dbl, ctypes.POINTER(GhbPhase), i32,
                             ctypes.POINTER(GhbOptions)]),
        "ghb_set_coeffs": (i32, [P, dbl, ctypes.POINTER(GhbPhase), i32]),
        "ghb_set_options": (i32, [P, ctypes.POINTER(GhbOptions)]),
        "ghb_set_stream": (i32, [P, P]),
        "ghb_get_grid": (i32, [P, ip, ip, ip, ctypes.POINTER(i64)]),
        "ghb_field_elems": (i64, [P]),
        "ghb_matvec": (i32, [P, i32, i32, i32, P, P, P]),
        "ghb_solve_primal": (i32, [P, dp, P, ctypes.POINTER(GhbSolveInfo)]),
        "ghb_solve_dual": (i32, [P, dp, P, ctypes.POINTER(GhbSolveInfo)]),
        "ghb_gram": (i32, [P, i32, i32, ctypes.POINTER(P), dp]),
        "ghb_bounds": (i32, [P, dp, dp, ctypes.POINTER(GhbSolveInfo)]),
        "ghb_table_elems": (i64, [P]),
        "ghb_grid_elems": (i64, [P]),
        "ghb_copy_table": (i32, [P, i32, P]),
        "ghb_copy_grid_values": (i32, [P, i32, P]),
        "ghb_device_bytes": (i64, [P]),
        "ghb_last_error": (ctypes.c_char_p, []),
        "ghb_destroy": (None, [P]),
        "ghb_version": (ctypes.c_char_p, []),
        "ghb_profile": (i32, [P, i32]),
        "ghb_batch_create": (i32, [ctypes.POINTER(P), ctypes.POINTER(GhbOptions), i64, i32]),
        "ghb_batch_submit": (i32, [P, i32, ip, dbl, ctypes.POINTER(GhbPhase), i32, ctypes.POINTER(i64)]),
        "ghb_batch_step": (i32, [P, i32, ip, ip]),
        "ghb_batch_run": (i32, [P, i32]),
        "ghb_batch_results": (i32, [P, ctypes.POINTER(GhbResult), i32]),
        "ghb_batch_stats": (i32, [P, ctypes.POINTER(i64), ip, ip, ctypes.POINTER(i64), ctypes.POINTER(i64)]),
        "ghb_batch_destroy": (None, [P]),
        "ghb_gram_noalloc": (i32, [i32, ip, ip, P, i32, ctypes.POINTER(P), dp, P]),
        "ghb_profile_read": (i32, [P, i32, ctypes.POINTER(i64), dp, dp, dp]),
        "ghb_tune_get": (i32, [i32, ip]),
        "ghb_tune_set": (i32, [i32, ip]),
        "ghb_tune_reset": (i32, []),
        "ghb_bounds_gani": (i32, [P, dp, dp, dp, dp, ctypes.POINTER(GhbSolveInfo)]),
        "ghb_solve_ex": (i32, [P, i32, dp, P, P, ctypes.POINTER(GhbSolveInfo), dp, i32, ip]),
        "ghb_prolong": (i32, [i32, ip, P, ip, P, P]),
        "ghb_create_image": (i32, [ctypes.POINTER(P), i32, ip, ip, dp, ctypes.POINTER(GhbOptions)]),
        "ghb_set_image": (i32, [P, ip, dp]),
        "ghb_set_form": (i32, [P, i32]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(status):
    if status != GHB_OK:
        raise GhbError(status, _lib.ghb_last_error().decode())
    return status


def make_phases(inclusions):
    """ctypes array of GhbPhase from (shape, center, size, value) tuples."""
    n = len(inclusions)
    arr = (GhbPhase * max(n, 1))()
    for i, (shape, center, size, value) in enumerate(inclusions):
        arr[i].shape = int(shape)
        for a in range(3):
            arr[i].center[a] = float(center[a]) if a < len(center) else 0.0
            arr[i].size[a] = float(size[a]) if a < len(size) else 0.0
        arr[i].value = float(value)
    return arr, n


@dataclass
class Options:
    tol: float = 1e-10
    max_iter: int = 20000
    precision: str = "fp64"          # "fp64" or "mixed"
    inner_tol: float = 1e-5
    max_outer: int = 20
    M: tuple = (0, 0, 0)

    def to_c(self):
        o = GhbOptions()
        load_library().ghb_default_options(ctypes.byref(o))
        o.tol = self.tol
        o.max_iter = self.max_iter
        o.precision = {"fp64": GHB_FP64, "mixed": GHB_MIXED}[self.precision]
        o.inner_tol = self.inner_tol
        o.max_outer = self.max_outer
        for a in range(3):
            o.M[a] = int(self.M[a]) if a < len(self.M) else 0
        return o


class Context:
    """One microstructure at one order N on the current CUDA device (C ABI ghb_ctx)."""

    def __init__(self, d, N, a0, inclusions, **options):
        lib = load_library()
        self.d = int(d)
        self.opts = Options(**options)
        Nc = (ctypes.c_int * 3)(*([int(n) for n in N] + [1] * (3 - len(N))))
        ph, n = make_phases(inclusions)
        self._h = ctypes.c_void_p()
        opt = self.opts.to_c()
        _check(lib.ghb_create(ctypes.byref(self._h), self.d, Nc, float(a0), ph, n, ctypes.byref(opt)))
        dd = ctypes.c_int()
        Nn = (ctypes.c_int * 3)()
        Mm = (ctypes.c_int * 3)()
        fe = ctypes.c_int64()
        _check(lib.ghb_get_grid(self._h, ctypes.byref(dd), Nn, Mm, ctypes.byref(fe)))
        self.N = [Nn[a] for a in range(self.d)]
        self.M = [Mm[a] for a in range(self.d)]
        self.field_elems = fe.value
        self.h = (self.N[-1] + 1) // 2

    @classmethod
    def from_microstructure(cls, m: dict, **options):
        return cls(m["d"], m["N"], m["a0"], m["inclusions"], **options)

    @classmethod
    def from_image(cls, image, N, **options):
        """A context whose coefficient is the piecewise-constant pixel image
        `image` (numpy array of shape P, positive values; ghb_create_image)."""
        img = np.ascontiguousarray(np.asarray(image, dtype=np.float64))
        d = img.ndim
        ctx = cls(d, N, 1.0, [], **options)
        ctx.set_image(img)
        return ctx

    def set_form(self, form):
        """"double_grid" (Algorithm 2) or "reduced" (Algorithm 3, needs M = 2N)."""
        f = {"double_grid": GHB_FORM_DOUBLE_GRID, "reduced": GHB_FORM_REDUCED}[form]
        _check(_lib.ghb_set_form(self._h, f))

    def set_image(self, image):
        """Replace the coefficient by a pixel image (ghb_set_image)."""
        img = np.ascontiguousarray(np.asarray(image, dtype=np.float64))
        P = (ctypes.c_int * 3)(*(list(img.shape) + [1] * (3 - img.ndim)))
        _check(_lib.ghb_set_image(self._h, P, img.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))

    # -- lifetime -----------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            _lib.ghb_destroy(self._h)
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

    # -- configuration --------------------------------------------------------
    @property
    def field_shape(self):
        """Shape of one half-spectrum field: (d, N_1, .., N_{d-1}, (N_d+1)/2)."""
        return (self.d, *self.N[:-1], self.h)

    def set_coeffs(self, a0, inclusions):
        ph, n = make_phases(inclusions)
        _check(_lib.ghb_set_coeffs(self._h, float(a0), ph, n))

    def set_options(self, **options):
        for k, v in options.items():
            setattr(self.opts, k, v)
        o = self.opts.to_c()
        _check(_lib.ghb_set_options(self._h, ctypes.byref(o)))

    def set_stream(self, stream):
        """Use a torch.cuda.Stream (or None for the context's own stream)."""
        ptr = None if stream is None else stream.cuda_stream
        _check(_lib.ghb_set_stream(self._h, ptr))

    def device_bytes(self):
        return int(_lib.ghb_device_bytes(self._h))

    def profile(self, enable=True):
        _check(_lib.ghb_profile(self._h, int(bool(enable))))

    def profile_read(self):
        """{class name + ('_f32'|'_f64'): dict(launches, ms, bytes, flops)} of the recorded launches."""
        out = {}
        for k, name in enumerate(PROFILE_CLASSES):
            for f in (0, 1):
                n = ctypes.c_int64()
                ms, b, fl = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
                _check(_lib.ghb_profile_read(self._h, 2 * k + f, ctypes.byref(n), ctypes.byref(ms),
                                             ctypes.byref(b), ctypes.byref(fl)))
                if n.value:
                    out[name + ("_f32" if f else "_f64")] = dict(launches=n.value, ms=ms.value, bytes=b.value,
                                                                  flops=fl.value)
        return out

    # -- operator -------------------------------------------------------------
    def matvec(self, x, kind=GHB_PRIMAL, project=True, out=None, stream=None):
        """y = G A^full x on the device for a half-spectrum field x (torch
        complex128 -> FP64 operator, complex64 -> FP32 operator)."""
        import torch
        if x.dtype == torch.complex128:
            prec = GHB_FP64
        elif x.dtype == torch.complex64:
            prec = GHB_FP32
        else:
            raise TypeError("x must be complex128 or complex64")
        if tuple(x.shape) != self.field_shape or not x.is_cuda or not x.is_contiguous():
            raise ValueError(f"x must be a contiguous CUDA tensor of shape {self.field_shape}")
        y = torch.empty_like(x) if out is None else out
        handle = (stream if stream is not None else torch.cuda.current_stream()).cuda_stream
        # handle 0 is the legacy default stream; the C ABI reads NULL as "the
        # context's own stream", so name the legacy stream explicitly (0x1)
        s = ctypes.c_void_p(handle if handle != 0 else 1)
        _check(_lib.ghb_matvec(self._h, int(kind), prec, int(bool(project)), ctypes.c_void_p(x.data_ptr()),
                               ctypes.c_void_p(y.data_ptr()), s))
        return y

    # -- solves ---------------------------------------------------------------
    def solve(self, kind, E, want_field=False):
        """Minimiser for load E; returns (info dict, field or None).  A status of
        GHB_ERR_NOT_CONVERGED is reported in info, not raised."""
        import torch
        Ec = (ctypes.c_double * 3)(*([float(e) for e in E] + [0.0] * (3 - len(E))))
        field = torch.empty(self.field_shape, dtype=torch.complex128, device="cuda") if want_field else None
        inf = GhbSolveInfo()
        fn = _lib.ghb_solve_primal if kind == GHB_PRIMAL else _lib.ghb_solve_dual
        st = fn(self._h, Ec, ctypes.c_void_p(field.data_ptr()) if want_field else None, ctypes.byref(inf))
        if st not in (GHB_OK, GHB_ERR_NOT_CONVERGED):
            _check(st)
        return inf.as_dict(), field

    def gram(self, kind, fields):
        ptrs = (ctypes.c_void_p * 3)(*[f.data_ptr() for f in fields])
        out = (ctypes.c_double * 9)()
        _check(_lib.ghb_gram(self._h, int(kind), len(fields), ptrs, out))
        m = len(fields)
        return np.array(out[: m * m]).reshape(m, m)

    def bounds(self):
        """(upper, lower, infos): the d x d Ga bounds and 2d solve records."""
        d = self.d
        up = (ctypes.c_double * 9)()
        lo = (ctypes.c_double * 9)()
        infos = (GhbSolveInfo * 6)()
        st = _lib.ghb_bounds(self._h, up, lo, infos)
        if st not in (GHB_OK, GHB_ERR_NOT_CONVERGED):
            _check(st)
        U = np.array(up[: d * d]).reshape(d, d)
        L = np.array(lo[: d * d]).reshape(d, d)
        return U, L, [infos[i].as_dict() for i in range(2 * d)], st

    def solve_ex(self, E, kind=GHB_PRIMAL, x0=None, energies=False, max_energies=100000):
        """One solve (ghb_solve_ex): returns (field, info, energies, status); field
        is the admissible E + e as a complex128 CUDA tensor of the half-spectrum
        shape; x0: initial fluctuation (complex128 CUDA tensor or None);
        energies: the energy along the iterates (bound tracking) when True."""
        import torch
        d = self.d
        Ec = (ctypes.c_double * 3)(*([float(v) for v in E] + [0.0] * (3 - len(E))))
        out = torch.empty(self.field_shape, dtype=torch.complex128, device="cuda")
        info = GhbSolveInfo()
        buf = (ctypes.c_double * max_energies)() if energies else None
        n = ctypes.c_int(0)
        x0p = None if x0 is None else ctypes.c_void_p(x0.contiguous().data_ptr())
        torch.cuda.synchronize()
        st = _lib.ghb_solve_ex(self._h, int(kind), Ec, x0p, ctypes.c_void_p(out.data_ptr()), ctypes.byref(info),
                               buf, int(max_energies) if energies else 0, ctypes.byref(n))
        if st not in (GHB_OK, GHB_ERR_NOT_CONVERGED):
            _check(st)
        hist = np.array(buf[: n.value]) if energies else None
        return out, info.as_dict(), hist, st

    def bounds_gani(self):
        """(upper, lower, A_gani, B_gani_inv, infos, status): the a-posteriori
        guaranteed bounds of the GaNi scheme (exact energies of the GaNi
        minimisers, eq. GaNi_apost) and the GaNi matrices (ghb_bounds_gani)."""
        d = self.d
        bufs = [(ctypes.c_double * 9)() for _ in range(4)]
        infos = (GhbSolveInfo * 6)()
        st = _lib.ghb_bounds_gani(self._h, *bufs, infos)
        if st not in (GHB_OK, GHB_ERR_NOT_CONVERGED):
            _check(st)
        mats = [np.array(b[: d * d]).reshape(d, d) for b in bufs]
        return (*mats, [infos[i].as_dict() for i in range(2 * d)], st)

    # -- data for checks --------------------------------------------------------
    def table(self, kind=GHB_PRIMAL):
        """a^ (or (1/a)^) on Z_{2N-1}, half spectrum, as a complex128 CUDA tensor."""
        import torch
        shape = tuple(2 * n - 1 for n in self.N[:-1]) + (self.N[-1],)
        t = torch.empty(shape, dtype=torch.complex128, device="cuda")
        _check(_lib.ghb_copy_table(self._h, int(kind), ctypes.c_void_p(t.data_ptr())))
        return t

    def grid_values(self, kind=GHB_PRIMAL):
        """A_M (or B_M) on the double grid, float64 CUDA tensor of shape M."""
        import torch
        t = torch.empty(tuple(self.M), dtype=torch.float64, device="cuda")
        _check(_lib.ghb_copy_grid_values(self._h, int(kind), ctypes.c_void_p(t.data_ptr())))
        return t


def gram_noalloc(d, N, M, grid, fields, stream=None):
    """ghb_gram_noalloc: the Gram matrix of FP64 half-spectrum fields without any
    device allocation (scratch in a fixed 32 MiB device array; for callers that
    cannot allocate).  grid: FP64 CUDA tensor of the double-grid values (prod(M)
    entries); fields: 1..d complex128 CUDA tensors of d * N_1 ... N_{d-1} *
    (N_d + 1)/2 entries each, contiguous, on the current device."""
    import torch
    lib = load_library()
    d = int(d)
    if d not in (2, 3) or len(N) != d or len(M) != d:
        raise ValueError("d must be 2 or 3 with d orders N and d double-grid sizes M")
    if not 1 <= len(fields) <= d:
        raise ValueError(f"between 1 and d = {d} fields are allowed, got {len(fields)}")

    def check(t, dtype, n, what):
        ok = isinstance(t, torch.Tensor) and t.is_cuda
        if ok:
            dev = torch.cuda.current_device()
            ok = t.device.index == dev and t.dtype == dtype and t.is_contiguous() and t.numel() == n
        if not ok:
            raise ValueError(f"{what} must be a contiguous {dtype} tensor of {n} entries on the current CUDA device")

    check(grid, torch.float64, int(np.prod([int(m) for m in M])), "grid")
    nf = d * int(np.prod([int(n) for n in N[:-1]])) * ((int(N[-1]) + 1) // 2)
    for f in fields:
        check(f, torch.complex128, nf, "each field")
    Nc = (ctypes.c_int * 3)(*([int(n) for n in N] + [1] * (3 - len(N))))
    Mc = (ctypes.c_int * 3)(*([int(n) for n in M] + [1] * (3 - len(M))))
    ptrs = (ctypes.c_void_p * 3)(*[f.data_ptr() for f in fields])
    out = (ctypes.c_double * 9)()
    s = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
    _check(lib.ghb_gram_noalloc(d, Nc, Mc, ctypes.c_void_p(grid.data_ptr()), len(fields), ptrs, out, s))
    m = len(fields)
    return np.array(out[: m * m]).reshape(m, m)


def prolong(x, N_fine):
    """ghb_prolong: the half-spectrum field x (complex128 CUDA tensor of order
    N_coarse) as a field of order N_fine, the same trigonometric polynomial."""
    import torch
    d = x.shape[0]
    Nc = list(x.shape[1:-1]) + [2 * x.shape[-1] - 1]
    Nf = [int(n) for n in N_fine]
    out = torch.empty((d,) + tuple(Nf[:-1]) + ((Nf[-1] + 1) // 2,), dtype=torch.complex128, device=x.device)
    lib = load_library()
    a = (ctypes.c_int * 3)(*(Nc + [1] * (3 - d)))
    b = (ctypes.c_int * 3)(*(Nf + [1] * (3 - d)))
    torch.cuda.synchronize()
    _check(lib.ghb_prolong(d, a, ctypes.c_void_p(x.contiguous().data_ptr()), b, ctypes.c_void_p(out.data_ptr()), None))
    return out


TUNE_FIELDS = ["cap32", "tile32", "rows32", "ct_col", "ct_row", "cap64", "tile64"]


def tune_get(M):
    """Launch configuration of the transform passes for length M (ghb_tune_get;
    tunes M first if it has not been tuned in this process)."""
    lib = load_library()
    cfg = (ctypes.c_int * 7)()
    _check(lib.ghb_tune_get(int(M), cfg))
    return dict(zip(TUNE_FIELDS, list(cfg)))


def tune_set(M, **cfg):
    """Fix the configuration of length M (ghb_tune_set); fields not given keep
    their current values."""
    cur = tune_get(M)
    cur.update({k: int(v) for k, v in cfg.items()})
    arr = (ctypes.c_int * 7)(*[cur[k] for k in TUNE_FIELDS])
    _check(load_library().ghb_tune_set(int(M), arr))
    return cur


def tune_reset():
    """Forget every stored configuration (ghb_tune_reset)."""
    _check(load_library().ghb_tune_reset())


class Batch:
    """Many bound-pair requests solved together (C ABI ghb_batch_*): one launch
    per kernel and CG iteration over all active solves, continuous admission."""

    def __init__(self, budget_bytes=0, max_active=0, **options):
        lib = load_library()
        options.setdefault("precision", "mixed")
        self.opts = Options(**options)
        self._h = ctypes.c_void_p()
        o = self.opts.to_c()
        _check(lib.ghb_batch_create(ctypes.byref(self._h), ctypes.byref(o), int(budget_bytes), int(max_active)))
        self._buf = (GhbResult * 256)()

    def submit(self, m: dict) -> int:
        Nc = (ctypes.c_int * 3)(*([int(n) for n in m["N"]] + [1] * (3 - len(m["N"]))))
        ph, n = make_phases(m["inclusions"])
        rid = ctypes.c_int64()
        _check(_lib.ghb_batch_submit(self._h, int(m["d"]), Nc, float(m["a0"]), ph, n, ctypes.byref(rid)))
        return rid.value

    def step(self, iterations=8):
        a, p = ctypes.c_int(), ctypes.c_int()
        _check(_lib.ghb_batch_step(self._h, int(iterations), ctypes.byref(a), ctypes.byref(p)))
        return a.value, p.value

    def run(self, iterations=8):
        _check(_lib.ghb_batch_run(self._h, int(iterations)))

    def results(self):
        out = []
        while True:
            n = _lib.ghb_batch_results(self._h, self._buf, len(self._buf))
            out.extend(self._buf[i].as_dict() for i in range(n))
            if n < len(self._buf):
                return out

    def stats(self):
        b, f, L = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        a, p = ctypes.c_int(), ctypes.c_int()
        _check(_lib.ghb_batch_stats(self._h, ctypes.byref(b), ctypes.byref(a), ctypes.byref(p), ctypes.byref(f),
                                    ctypes.byref(L)))
        return {"bytes_in_use": b.value, "active": a.value, "pending": p.value, "finished": f.value,
                "launches": L.value}

    def close(self):
        if getattr(self, "_h", None):
            _lib.ghb_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# layout helpers (index permutations and conjugation only)
# ---------------------------------------------------------------------------
def half_from_full(x):
    """(d, N_1..N_d) centred full spectrum -> (d, N_1..N_{d-1}, (N_d+1)/2) half spectrum."""
    Nd = x.shape[-1]
    return x[..., (Nd - 1) // 2:]


def full_from_half(xh, Nd):
    """Inverse of half_from_full using x(-k) = conj x(k) (numpy arrays)."""
    xh = np.asarray(xh)
    d = xh.ndim - 1
    c = (Nd - 1) // 2
    out = np.zeros(xh.shape[:-1] + (Nd,), dtype=xh.dtype)
    out[..., c:] = xh
    # k_d < 0: x(k', -j) = conj x(-k', j) with k' mirrored on the leading axes
    mirrored = np.conj(xh[(slice(None),) + (slice(None, None, -1),) * (d - 1) + (slice(1, None),)])
    out[..., :c] = mirrored[..., ::-1]
    return out
