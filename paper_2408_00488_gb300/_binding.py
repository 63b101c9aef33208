"""ctypes binding of libcsl.so (include/csl.h).  Argument marshalling only:
every step of the solve runs in the library's CUDA kernels.  Importing this
module loads the library and raises if it has not been built."""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Sequence, Tuple

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "libcsl.so")

OK, INVALID_ARG, UNSUPPORTED_SIZE, SINGULAR_PRECOND, BREAKDOWN, NOT_CONVERGED, TIMEOUT, CUDA_ERROR, \
    OUT_OF_MEMORY = range(9)
PREC_FP64, PREC_FP32, PREC_BF16X3, PREC_BF16X6, PREC_FP32_PRECOND = 0, 1, 2, 3, 4
_PREC = {"fp64": PREC_FP64, "fp32": PREC_FP32, "mixed": PREC_FP32, "bf16x3": PREC_BF16X3, "bf16x6": PREC_BF16X6,
         "fp32_precond": PREC_FP32_PRECOND}


class PlanOptions(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("gamma_override", ctypes.c_double),
                ("lines_per_cta", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("autotune", ctypes.c_int), ("programmatic_launch", ctypes.c_int),
                ("float_pair_stencil", ctypes.c_int), ("update_mode", ctypes.c_int),
                ("body_iters", ctypes.c_int), ("warm_start", ctypes.c_int), ("history", ctypes.c_int),
                ("reserved", ctypes.c_int * 1)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("status", ctypes.c_int), ("relres", ctypes.c_double),
                ("pnorm", ctypes.c_double), ("gamma", ctypes.c_double), ("checks", ctypes.c_int),
                ("launches", ctypes.c_int), ("reserved", ctypes.c_int * 6)]


class SystemDesc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int64 * 3), ("coef_faces", ctypes.c_void_p * 3),
                ("alpha", ctypes.c_double), ("beta", ctypes.c_double)]


# name -> (restype, argtypes)
_P = ctypes.c_void_p
class ParaDiagInfo(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int), ("status", ctypes.c_int), ("relres", ctypes.c_double),
                ("inner_iters_max", ctypes.c_int), ("reserved", ctypes.c_int * 5)]


class HelmholtzInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("status", ctypes.c_int), ("relres", ctypes.c_double),
                ("inner_iters_total", ctypes.c_int), ("restarts", ctypes.c_int), ("reserved", ctypes.c_int * 4)]


_SIGS = {
    "csl_helmholtz_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                            ctypes.POINTER(_P), ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_int, ctypes.POINTER(PlanOptions), _P]),
    "csl_helmholtz_solve": (ctypes.c_int, [_P, _P, _P, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_int, ctypes.POINTER(HelmholtzInfo)]),
    "csl_helmholtz_destroy": (None, [_P]),
    "csl_paradiag_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                           ctypes.POINTER(_P), ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                           ctypes.POINTER(PlanOptions), _P]),
    "csl_paradiag_solve": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                          ctypes.c_int, ctypes.POINTER(ParaDiagInfo)]),
    "csl_paradiag_destroy": (None, [_P]),
    "csl_test_convert_d2f": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P]),
    "csl_test_convert_f2d": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P]),
    "csl_probe_sync_cost": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "csl_version": (ctypes.c_char_p, []),
    "csl_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "csl_last_error": (ctypes.c_char_p, []),
    "csl_plan_options_init": (ctypes.c_int, [ctypes.POINTER(PlanOptions)]),
    "csl_plan_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(_P), ctypes.c_double, ctypes.c_double,
                                       ctypes.POINTER(PlanOptions), _P]),
    "csl_plan_destroy": (None, [_P]),
    "csl_plan_set_stream": (ctypes.c_int, [_P, _P]),
    "csl_plan_workspace_bytes": (ctypes.c_size_t, [_P]),
    "csl_plan_gamma": (ctypes.c_double, [_P]),
    "csl_plan_config": (ctypes.c_char_p, [_P]),
    "csl_apply": (ctypes.c_int, [_P, _P, _P]),
    "csl_precondition": (ctypes.c_int, [_P, _P, _P]),
    "csl_solve": (ctypes.c_int, [_P, _P, _P, ctypes.c_double, ctypes.c_int, ctypes.POINTER(SolveInfo)]),
    "csl_solve_host": (ctypes.c_int, [_P, _P, _P, ctypes.c_double, ctypes.c_int, ctypes.POINTER(SolveInfo)]),
    "csl_solve_history": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_int)]),
    "csl_adjoint": (ctypes.c_int, [_P, _P, _P, ctypes.c_double, ctypes.c_int, ctypes.POINTER(SolveInfo)]),
    "csl_coef_grad": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(_P)]),
    "csl_precondition_static": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.c_double,
                                               ctypes.c_double, ctypes.c_double, ctypes.c_int, _P, _P, _P]),
    "csl_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(SystemDesc),
                                        ctypes.POINTER(PlanOptions), _P]),
    "csl_batch_solve": (ctypes.c_int, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.c_double, ctypes.c_int,
                                       ctypes.POINTER(SolveInfo)]),
    "csl_batch_destroy": (None, [_P]),
    "csl_batch_workspace_bytes": (ctypes.c_size_t, [_P]),
    "csl_tune_cache_save": (ctypes.c_int, [ctypes.c_char_p]),
    "csl_tune_cache_load": (ctypes.c_int, [ctypes.c_char_p]),
    "csl_time_kernels": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_int)]),
}


def load_library(path: str = LIBPATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"libcsl.so not found at {path}: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'` "
                          "(there is no fallback implementation)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = load_library()


class CSLError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        detail = lib.csl_last_error().decode() if status in (CUDA_ERROR, OUT_OF_MEMORY) else ""
        super().__init__(f"{where}: {status_string(status)}" + (f" [{detail}]" if detail else ""))


def status_string(status: int) -> str:
    return lib.csl_status_string(int(status)).decode()


def version() -> str:
    return lib.csl_version().decode()


def _check(status: int, where: str, allow=(OK,)):
    if status not in allow:
        raise CSLError(status, where)
    return status


@dataclass
class Info:
    iters: int
    status: int
    relres: float
    pnorm: float
    gamma: float
    checks: int
    launches: int

    @property
    def converged(self) -> bool:
        return self.status == OK

    @staticmethod
    def from_c(ci: SolveInfo) -> "Info":
        return Info(ci.iters, ci.status, ci.relres, ci.pnorm, ci.gamma, ci.checks, ci.launches)


def _torch():
    import torch
    return torch


def _stream_handle(stream=None) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _dptr(t, dtype_names, what: str) -> int:
    if not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if str(t.dtype).replace("torch.", "") not in dtype_names:
        raise ValueError(f"{what} must have dtype in {dtype_names}, got {t.dtype}")
    return t.data_ptr()


class Plan:
    """A solver plan for one grid, coefficient field and shift lambda.

    faces: (x-faces, y-faces[, z-faces]) float64 CUDA tensors in the layout of
    include/csl.h (x fastest).  precision: "fp64", "fp32" (FP32 sine
    transforms and scale inside P^{-1}; everything else FP64), or "bf16x3" /
    "bf16x6" (as "fp32", with the y and z transforms of lines of 32, 64 or
    128 points as split-bf16 tensor-core GEMMs, 3 or 6 products).
    """

    def __init__(self, faces: Sequence, lam: complex, precision: str = "fp64",
                 gamma: Optional[float] = None, lines_per_cta: int = 0, use_graph: bool = True,
                 autotune: bool = True, stream=None, programmatic_launch: bool = True,
                 float_pair_stencil: bool = True, update_mode: int = 0, body_iters: int = 0,
                 warm_start: bool = False, history: int = 0):
        torch = _torch()
        dim = len(faces)
        if dim not in (2, 3):
            raise ValueError("dim must be 2 or 3")
        fx = faces[0]
        nx = fx.shape[-1] - 1
        ny = fx.shape[-2]
        nz = fx.shape[-3] if dim == 3 else 1
        self.dim = dim
        self.shape = (ny, nx) if dim == 2 else (nz, ny, nx)
        self.M = nx * ny * nz
        self.lam = complex(lam)
        self._faces = [f.contiguous() for f in faces]
        for i, f in enumerate(self._faces):
            _dptr(f, ("float64",), f"faces[{i}]")
        n = (ctypes.c_int64 * 3)(nx, ny, nz)
        ptrs = (_P * 3)(*([f.data_ptr() for f in self._faces] + [None] * (3 - dim)))
        opt = PlanOptions()
        lib.csl_plan_options_init(ctypes.byref(opt))
        opt.precision = _PREC[precision]
        opt.gamma_override = float(gamma) if gamma is not None else float("nan")
        opt.lines_per_cta = int(lines_per_cta)
        opt.use_graph = 1 if use_graph else 0
        opt.autotune = 1 if autotune else 0
        opt.programmatic_launch = 1 if programmatic_launch else 0
        opt.float_pair_stencil = 1 if float_pair_stencil else 0
        opt.update_mode = int(update_mode)
        opt.body_iters = int(body_iters)
        opt.warm_start = 1 if warm_start else 0
        opt.history = int(history)
        self.warm_start = bool(warm_start)
        self.precision = precision
        h = _P()
        st = lib.csl_plan_create(ctypes.byref(h), dim, n, ptrs, self.lam.real, self.lam.imag,
                                 ctypes.byref(opt), _stream_handle(stream))
        _check(st, "csl_plan_create")
        self._h = h
        self._faces = None  # the plan keeps its own copy

    # -- lifetime ------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            lib.csl_plan_destroy(self._h)
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

    def _sync_stream(self, stream=None):
        lib.csl_plan_set_stream(self._h, _stream_handle(stream))

    @property
    def gamma(self) -> float:
        return lib.csl_plan_gamma(self._h)

    @property
    def config(self) -> str:
        """Launch configuration chosen for this plan (autotuned or default)."""
        return lib.csl_plan_config(self._h).decode()

    @property
    def workspace_bytes(self) -> int:
        return lib.csl_plan_workspace_bytes(self._h)

    # -- operations ----------------------------------------------------------
    def _check_grid(self, t, what: str, pairs_ok: bool = False):
        """The library reads and writes whole grid vectors through plain
        pointers, so every tensor passed must hold exactly one grid vector."""
        shape = _grid_vector(t, what) if pairs_ok else tuple(t.shape)
        if int(np.prod(shape)) != self.M:
            raise ValueError(f"{what} must hold one grid vector of {self.M} points (grid {self.shape}), "
                             f"got shape {tuple(t.shape)}")

    def apply(self, z):
        """(K + lambda I) z for a complex128 CUDA tensor of the grid's shape."""
        torch = _torch()
        self._check_grid(z, "z")
        self._sync_stream()
        out = torch.empty_like(z)
        _check(lib.csl_apply(self._h, _dptr(z, ("complex128",), "z"), out.data_ptr()), "csl_apply")
        return out

    def precondition(self, v):
        """P^{-1} v for a complex128 (or (...,2) float64) CUDA tensor."""
        torch = _torch()
        self._check_grid(v, "v", pairs_ok=True)
        self._sync_stream()
        out = torch.empty_like(v)
        _check(lib.csl_precondition(self._h, _dptr(v, ("complex128", "float64"), "v"), out.data_ptr()),
               "csl_precondition")
        return out

    def solve(self, f, tol: float = 1e-8, maxit: int = 1000, out=None, x0=None) -> Tuple[object, Info]:
        """Solve (K + lambda I) z = f.  x0 (plans made with warm_start=True):
        the initial guess, copied into the output before the call (the
        library reads the output vector as x0)."""
        torch = _torch()
        self._check_grid(f, "f")
        if out is not None:
            self._check_grid(out, "out")
        self._sync_stream()
        z = torch.empty_like(f) if out is None else out
        if self.warm_start:
            if x0 is None:
                z.zero_()
            elif x0 is not z:
                self._check_grid(x0, "x0")
                z.copy_(x0)
        elif x0 is not None:
            raise ValueError("x0 needs a plan made with warm_start=True")
        ci = SolveInfo()
        st = lib.csl_solve(self._h, _dptr(f, ("complex128",), "f"), _dptr(z, ("complex128",), "z"),
                           float(tol), int(maxit), ctypes.byref(ci))
        _check(st, "csl_solve", allow=(OK, NOT_CONVERGED, BREAKDOWN))
        return z, Info.from_c(ci)

    def adjoint(self, g, tol: float = 1e-8, maxit: int = 1000, out=None):
        torch = _torch()
        self._check_grid(g, "g")
        if out is not None:
            self._check_grid(out, "out")
        self._sync_stream()
        y = torch.empty_like(g) if out is None else out
        if self.warm_start and out is None:
            y.zero_()  # no initial guess given: start from 0
        ci = SolveInfo()
        st = lib.csl_adjoint(self._h, _dptr(g, ("complex128",), "g"), _dptr(y, ("complex128",), "y"),
                             float(tol), int(maxit), ctypes.byref(ci))
        _check(st, "csl_adjoint", allow=(OK, NOT_CONVERGED, BREAKDOWN))
        return y, Info.from_c(ci)

    def solve_host(self, f_host, z_host, tol: float = 1e-8, maxit: int = 1000) -> Info:
        """Solve with host (CPU, ideally pinned) complex128 tensors/arrays."""
        for t, what in ((f_host, "f_host"), (z_host, "z_host")):
            if int(np.prod(tuple(t.shape))) != self.M or "complex128" not in str(t.dtype):
                raise ValueError(f"{what} must be a complex128 host array of {self.M} points")
        self._sync_stream()
        ci = SolveInfo()
        fp = f_host.data_ptr() if hasattr(f_host, "data_ptr") else f_host.ctypes.data
        zp = z_host.data_ptr() if hasattr(z_host, "data_ptr") else z_host.ctypes.data
        st = lib.csl_solve_host(self._h, fp, zp, float(tol), int(maxit), ctypes.byref(ci))
        _check(st, "csl_solve_host", allow=(OK, NOT_CONVERGED, BREAKDOWN))
        return Info.from_c(ci)

    def history(self, cap: int = 100000):
        """|eta_j| / |eta_0| of each iteration of the last solve (plans made
        with history > 0): the MINRES residual estimate in the P^{-1}-norm."""
        buf = (ctypes.c_double * max(1, int(cap)))()
        cnt = ctypes.c_int(0)
        _check(lib.csl_solve_history(self._h, buf, int(cap), ctypes.byref(cnt)), "csl_solve_history")
        return [buf[i] for i in range(cnt.value)]

    def time_kernels(self, reps: int = 10):
        """{kernel name: mean ms per launch} for the kernels of one iteration
        (measurement hook; run a solve first so the vectors hold real data)."""
        self._sync_stream()
        ms = (ctypes.c_double * 8)()
        names = (ctypes.c_char_p * 8)()
        cnt = ctypes.c_int(0)
        _check(lib.csl_time_kernels(self._h, int(reps), ms, names, ctypes.byref(cnt)), "csl_time_kernels")
        out = []
        for i in range(cnt.value):
            out.append((names[i].decode(), ms[i]))
        return out

    def coef_grad(self, z, y):
        torch = _torch()
        self._check_grid(z, "z")
        self._check_grid(y, "y")
        self._sync_stream()
        nz, ny, nx = (1,) + self.shape if self.dim == 2 else self.shape
        shapes = [(nz, ny, nx + 1), (nz, ny + 1, nx), (nz + 1, ny, nx)][: self.dim]
        grads = [torch.empty(s, dtype=torch.float64, device=z.device) for s in shapes]
        if self.dim == 2:
            grads = [g.reshape(s[1:]) for g, s in zip(grads, shapes)]
        ptrs = (_P * 3)(*([g.data_ptr() for g in grads] + [None] * (3 - self.dim)))
        _check(lib.csl_coef_grad(self._h, _dptr(z, ("complex128",), "z"), _dptr(y, ("complex128",), "y"),
                                 ptrs), "csl_coef_grad")
        return tuple(grads)


class Batch:
    """Many systems solved together (csl_batch_*): systems is a list of
    (faces, lam) with faces as for Plan; all systems share dim and precision."""

    def __init__(self, systems, precision: str = "fp64", autotune: bool = True, stream=None):
        self.n = len(systems)
        descs = (SystemDesc * self.n)()
        self._keep = []
        self.shapes = []
        for i, (faces, lam) in enumerate(systems):
            faces = [f.contiguous() for f in faces]
            self._keep.append(faces)
            dim = len(faces)
            nx = faces[0].shape[-1] - 1
            ny = faces[0].shape[-2]
            nz = faces[0].shape[-3] if dim == 3 else 1
            self.shapes.append((ny, nx) if dim == 2 else (nz, ny, nx))
            descs[i].dim = dim
            descs[i].n[0], descs[i].n[1], descs[i].n[2] = nx, ny, nz
            for d in range(3):
                descs[i].coef_faces[d] = _dptr(faces[d], ("float64",), "faces") if d < dim else None
            lam = complex(lam)
            descs[i].alpha, descs[i].beta = lam.real, lam.imag
        opt = PlanOptions()
        lib.csl_plan_options_init(ctypes.byref(opt))
        opt.precision = _PREC[precision]
        opt.autotune = 1 if autotune else 0
        h = _P()
        _check(lib.csl_batch_create(ctypes.byref(h), self.n, descs, ctypes.byref(opt), _stream_handle(stream)),
               "csl_batch_create")
        self._h = h
        self._keep = None

    def close(self):
        if getattr(self, "_h", None):
            lib.csl_batch_destroy(self._h)
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

    def solve(self, fs, tol: float = 1e-8, maxit: int = 1000, outs=None):
        torch = _torch()
        if len(fs) != self.n or (outs is not None and len(outs) != self.n):
            raise ValueError(f"one right-hand side (and output) per system: {self.n}")
        for i, shp in enumerate(self.shapes):
            for t in [fs[i]] + ([outs[i]] if outs is not None else []):
                if int(np.prod(tuple(t.shape))) != int(np.prod(shp)):
                    raise ValueError(f"system {i}: a vector of grid {shp} expected, got shape {tuple(t.shape)}")
        zs = [torch.empty_like(f) for f in fs] if outs is None else outs
        fp = (_P * self.n)(*[_dptr(f, ("complex128",), "f") for f in fs])
        zp = (_P * self.n)(*[_dptr(z, ("complex128",), "z") for z in zs])
        infos = (SolveInfo * self.n)()
        st = lib.csl_batch_solve(self._h, fp, zp, float(tol), int(maxit), infos)
        _check(st, "csl_batch_solve", allow=(OK, NOT_CONVERGED, BREAKDOWN))
        return zs, [Info.from_c(infos[i]) for i in range(self.n)]


def tune_cache_save(path: str) -> None:
    """Write the autotuner's shapes tuned so far in this process to `path`."""
    _check(lib.csl_tune_cache_save(os.fsencode(path)), "csl_tune_cache_save")


def tune_cache_load(path: str) -> None:
    """Merge the shapes of a file written by tune_cache_save into the
    autotuner's cache (plans created afterwards take them without timing)."""
    _check(lib.csl_tune_cache_load(os.fsencode(path)), "csl_tune_cache_load")


def _grid_vector(v, what: str):
    """The grid shape of a vector passed as complex128 (grid shape) or as
    float64 block pairs (grid shape + (2,))."""
    name = str(v.dtype).replace("torch.", "")
    if name == "complex128":
        return tuple(v.shape)
    if name == "float64":
        if v.dim() < 1 or v.shape[-1] != 2:
            raise ValueError(f"{what}: a float64 vector holds block pairs and needs a trailing dimension of 2, "
                             f"got shape {tuple(v.shape)}")
        return tuple(v.shape[:-1])
    raise ValueError(f"{what} must be complex128 or float64 block pairs, got {v.dtype}")


def precondition_static(v, gamma: float, lam: complex, precision: str = "fp64", out=None, stream=None):
    """P^{-1} v without a plan and without any device allocation by the
    library (csl_precondition_static): for callers that cannot allocate device
    memory themselves.  v: complex128 CUDA tensor of the grid's shape (2D or
    3D, at most 262144 points), or float64 block pairs of shape grid + (2,);
    gamma: the averaged coefficient of P; lam: the shift.  `out` (same shape,
    dtype and device as v) receives the result; without it one is allocated
    here by PyTorch."""
    torch = _torch()
    shape = _grid_vector(v, "v")
    dim = len(shape)
    if dim not in (2, 3):
        raise ValueError(f"v must describe a 2D or 3D grid, got grid shape {shape}")
    if out is None:
        y = torch.empty_like(v)
    else:
        if tuple(out.shape) != tuple(v.shape) or out.dtype != v.dtype:
            raise ValueError(f"out must have v's shape {tuple(v.shape)} and dtype {v.dtype}")
        if out.device != v.device:
            raise ValueError("out must be on v's device")
        y = out
    n = (ctypes.c_int64 * 3)(*(list(reversed(shape)) + [1] * (3 - dim)))
    lam = complex(lam)
    with torch.cuda.device(v.device):
        sh = _stream_handle(stream if stream is not None else torch.cuda.current_stream(v.device))
        st = lib.csl_precondition_static(dim, n, float(gamma), lam.real, lam.imag, _PREC[precision],
                                         _dptr(v, ("complex128", "float64"), "v"),
                                         _dptr(y, ("complex128", "float64"), "out"), sh)
    _check(st, "csl_precondition_static")
    return y


def test_convert(x, out_dtype, stream=None):
    """Test hook (include/csl_testing.h): the FP32-form kernels' integer-field
    conversion of a float64 CUDA tensor to float32 (round to nearest even) or
    of a float32 tensor to float64."""
    torch = _torch()
    x = x.contiguous()
    out = torch.empty(x.shape, dtype=out_dtype, device=x.device)
    if x.dtype == torch.float64 and out_dtype == torch.float32:
        st = lib.csl_test_convert_d2f(x.data_ptr(), out.data_ptr(), x.numel(), _stream_handle(stream))
    elif x.dtype == torch.float32 and out_dtype == torch.float64:
        st = lib.csl_test_convert_f2d(x.data_ptr(), out.data_ptr(), x.numel(), _stream_handle(stream))
    else:
        raise ValueError("float64 -> float32 or float32 -> float64")
    _check(st, "csl_test_convert")
    return out


def probe_sync_cost(kernels: int = 200, barriers: int = 1000, unreachable: bool = False):
    """Measurement hook (include/csl_testing.h): microseconds per kernel
    boundary of a CUDA graph of stage-shaped kernels with and without
    programmatic dependent launch, and per grid barrier of one cooperative
    kernel.  With unreachable=True every barrier wait runs out of its budget
    and CSLError(TIMEOUT) is raised."""
    out = (ctypes.c_double * 3)()
    st = lib.csl_probe_sync_cost(int(kernels), int(barriers), 1 if unreachable else 0, out)
    _check(st, "csl_probe_sync_cost")
    return {"graph_pdl_us": out[0], "graph_us": out[1], "grid_barrier_us": out[2]}


class ParaDiag:
    """All-at-once backward-Euler solve of u' + K u = g on L steps of size tau
    (csl_paradiag_*): preconditioned Richardson with the alpha-circulant time
    matrix, whose P^{-1} is a DFT in time plus L batched complex-shifted
    solves.  faces as for Plan; u0 a complex128 grid tensor, g a complex128
    tensor of shape (L, *grid)."""

    def __init__(self, faces, L: int, tau: float, a: float, precision: str = "fp64", autotune: bool = True,
                 stream=None):
        faces = [f.contiguous() for f in faces]
        dim = len(faces)
        nx = faces[0].shape[-1] - 1
        ny = faces[0].shape[-2]
        nz = faces[0].shape[-3] if dim == 3 else 1
        self.shape = (ny, nx) if dim == 2 else (nz, ny, nx)
        self.L = int(L)
        n = (ctypes.c_int64 * 3)(nx, ny, nz)
        fp = (_P * 3)(*[_dptr(faces[d], ("float64",), "faces") if d < dim else None for d in range(3)])
        opt = PlanOptions()
        lib.csl_plan_options_init(ctypes.byref(opt))
        opt.precision = _PREC[precision]
        opt.autotune = 1 if autotune else 0
        h = _P()
        _check(lib.csl_paradiag_create(ctypes.byref(h), dim, n, fp, self.L, float(tau), float(a), ctypes.byref(opt),
                                       _stream_handle(stream)), "csl_paradiag_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib.csl_paradiag_destroy(self._h)
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

    def solve(self, u0, g, tol: float = 1e-10, maxit: int = 20, inner_tol: float = 1e-12, inner_maxit: int = 2000,
              out=None):
        torch = _torch()
        if tuple(u0.shape) != self.shape or tuple(g.shape) != (self.L,) + self.shape:
            raise ValueError(f"u0 must have shape {self.shape} and g shape {(self.L,) + self.shape}")
        if out is not None and tuple(out.shape) != tuple(g.shape):
            raise ValueError("out must have g's shape")
        u = torch.empty_like(g) if out is None else out
        info = ParaDiagInfo()
        st = lib.csl_paradiag_solve(self._h, _dptr(u0.contiguous(), ("complex128",), "u0"),
                                    _dptr(g.contiguous(), ("complex128",), "g"), _dptr(u, ("complex128",), "u"),
                                    float(tol), int(maxit), float(inner_tol), int(inner_maxit), ctypes.byref(info))
        _check(st, "csl_paradiag_solve", allow=(OK, NOT_CONVERGED))
        return u, info


class Helmholtz:
    """Flexible GMRES for (K + lam I) u = f (e.g. lam = -k^2) preconditioned by
    the library's solve of (K + shift I) (csl_helmholtz_*)."""

    def __init__(self, faces, lam: complex, shift: complex, restart: int = 30, precision: str = "fp64",
                 autotune: bool = True, stream=None):
        faces = [f.contiguous() for f in faces]
        dim = len(faces)
        nx = faces[0].shape[-1] - 1
        ny = faces[0].shape[-2]
        nz = faces[0].shape[-3] if dim == 3 else 1
        self.shape = (ny, nx) if dim == 2 else (nz, ny, nx)
        n = (ctypes.c_int64 * 3)(nx, ny, nz)
        fp = (_P * 3)(*[_dptr(faces[d], ("float64",), "faces") if d < dim else None for d in range(3)])
        opt = PlanOptions()
        lib.csl_plan_options_init(ctypes.byref(opt))
        opt.precision = _PREC[precision]
        opt.autotune = 1 if autotune else 0
        lam, shift = complex(lam), complex(shift)
        h = _P()
        _check(lib.csl_helmholtz_create(ctypes.byref(h), dim, n, fp, lam.real, lam.imag, shift.real, shift.imag,
                                        int(restart), ctypes.byref(opt), _stream_handle(stream)),
               "csl_helmholtz_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib.csl_helmholtz_destroy(self._h)
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

    def solve(self, f, tol: float = 1e-8, maxit: int = 500, inner_tol: float = 1e-6, inner_maxit: int = 2000,
              out=None):
        torch = _torch()
        if tuple(f.shape) != self.shape or (out is not None and tuple(out.shape) != self.shape):
            raise ValueError(f"f (and out) must have the grid's shape {self.shape}")
        u = torch.empty_like(f) if out is None else out
        info = HelmholtzInfo()
        st = lib.csl_helmholtz_solve(self._h, _dptr(f.contiguous(), ("complex128",), "f"),
                                     _dptr(u, ("complex128",), "u"), float(tol), int(maxit), float(inner_tol),
                                     int(inner_maxit), ctypes.byref(info))
        _check(st, "csl_helmholtz_solve", allow=(OK, NOT_CONVERGED))
        return u, info

