"""Thin ctypes binding of ``libhzs.so`` (include/hzs.h).

Argument marshalling only: every step of a solve runs in the library's CUDA
kernels.  PyTorch provides device memory and the stream; tensors are passed as
raw device pointers.  The library must have been built (``build.build()``);
loading fails loudly otherwise, and nothing here falls back to a CPU path.
"""
from __future__ import annotations

import ctypes as ct
import os
from dataclasses import dataclass

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhzs.so")

# status codes
OK, NOT_CONVERGED = 0, 1
ERR_INVALID_ARG, ERR_CUDA, ERR_OOM = -1, -2, -3
ERR_SINGULAR_LOCAL, ERR_SINGULAR_COARSE, ERR_NONFINITE, ERR_TIMEOUT, ERR_BREAKDOWN = -4, -5, -6, -7, -8
# enums
DIRICHLET, SOMMERFELD = 0, 1
AS1, AS2, SAS2, SHS2 = 0, 1, 2, 3
COARSE_NONE, COARSE_P1, COARSE_B2 = 0, 1, 2
COARSE_SOLVER_AUTO, COARSE_SOLVER_DENSE, COARSE_SOLVER_BLOCK, COARSE_SOLVER_MULTILEVEL = 0, 1, 2, 3
FP64, MIXED = 0, 1

EXPORTS = (
    "hzs_grid_create", "hzs_grid_destroy", "hzs_precond_setup", "hzs_precond_destroy",
    "hzs_apply_operator", "hzs_apply_precond", "hzs_solve", "hzs_adjoint_solve",
    "hzs_kappa_gradient", "hzs_status_string", "hzs_last_error", "hzs_version",
    "hzs_apply_precond_noalloc", "hzs_solve_batched", "hzs_precond_get_info", "hzs_pipe_peaks",
)


class GridDesc(ct.Structure):
    _fields_ = [("n", ct.c_int), ("bc", ct.c_int), ("k", ct.c_double), ("kappa_dev", ct.c_void_p),
                ("nsub", ct.c_int), ("overlap", ct.c_int), ("nsub_y", ct.c_int)]


class PrecondDesc(ct.Structure):
    _fields_ = [("kind", ct.c_int), ("coarse", ct.c_int), ("coarse_ratio", ct.c_int),
                ("precision", ct.c_int), ("dedup_tiles", ct.c_int), ("coarse_solver", ct.c_int),
                ("autotune", ct.c_int), ("scaling_mode", ct.c_int), ("ml_nsub", ct.c_int), ("ml_overlap", ct.c_int),
                ("ml_ratio", ct.c_int)]


class PrecondInfo(ct.Structure):
    _fields_ = [("nfactors", ct.c_int), ("coarse_unknowns", ct.c_int), ("coarse_solver", ct.c_int),
                ("coarse_min_pivot", ct.c_double), ("tile_group", ct.c_int), ("tile_stages", ct.c_int),
                ("tile_threads_per_row", ct.c_int), ("autotuned", ct.c_int), ("apply_us_default", ct.c_double),
                ("apply_us_tuned", ct.c_double), ("coarse_tensor_cores", ct.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class PipeRates(ct.Structure):
    _fields_ = [("fp32_tflops", ct.c_double), ("fp32x2_tflops", ct.c_double), ("fp64_tflops", ct.c_double),
                ("int_tops", ct.c_double), ("cvt_tops", ct.c_double), ("mix_overlap", ct.c_double),
                ("sms", ct.c_int), ("clock_mhz", ct.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


SCALING_OWNER, SCALING_MULTIPLICITY = 0, 1
SOLVE_PROFILE = 1
SOLVE_ORTH_FP64 = 2
SOLVE_BASIS_WIDE = 4
SOLVE_GRAPH = 8
SOLVE_BASIS_DF = 16
SOLVE_ORTH_DFMA = 32
ORTH_CGS2_FP64, ORTH_DCGS2_FP64, ORTH_DCGS2_DF, ORTH_DCGS2_DFMA = 0, 1, 2, 3


class SolveDesc(ct.Structure):
    _fields_ = [("tol", ct.c_double), ("maxit", ct.c_int), ("flags", ct.c_int)]


class SolveInfo(ct.Structure):
    _fields_ = [("iterations", ct.c_int), ("converged", ct.c_int), ("relres_est", ct.c_double),
                ("relres_true", ct.c_double), ("t_solve_ms", ct.c_double), ("t_precond_ms", ct.c_double),
                ("t_matvec_ms", ct.c_double), ("t_orth_ms", ct.c_double), ("t_orth_dot_ms", ct.c_double),
                ("t_orth_update_ms", ct.c_double), ("launches", ct.c_longlong),
                ("basis_bits", ct.c_int), ("orth_kind", ct.c_int), ("status", ct.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class HzsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"hzs status {status}: {msg}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH) -> ct.CDLL:
    """Loads libhzs.so and declares the prototypes of every exported call."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2408_03571_gb300.build.build()")
    lib = ct.CDLL(path)
    P = ct.c_void_p
    lib.hzs_grid_create.argtypes = [ct.POINTER(GridDesc), P, ct.POINTER(P)]
    lib.hzs_grid_destroy.argtypes = [P]
    lib.hzs_grid_destroy.restype = None
    lib.hzs_precond_setup.argtypes = [P, ct.POINTER(PrecondDesc), ct.POINTER(P)]
    lib.hzs_precond_destroy.argtypes = [P]
    lib.hzs_precond_destroy.restype = None
    lib.hzs_apply_operator.argtypes = [P, P, P, ct.c_int]
    lib.hzs_apply_precond.argtypes = [P, P, P, ct.c_int]
    lib.hzs_apply_precond_noalloc.argtypes = [P, P, P, ct.c_int]
    lib.hzs_solve.argtypes = [P, ct.POINTER(SolveDesc), P, P, ct.c_int, ct.POINTER(SolveInfo)]
    lib.hzs_adjoint_solve.argtypes = [P, ct.POINTER(SolveDesc), P, P, ct.c_int, ct.POINTER(SolveInfo)]
    lib.hzs_solve_batched.argtypes = [ct.c_int, ct.POINTER(P), ct.POINTER(SolveDesc), ct.POINTER(P), ct.POINTER(P),
                                      ct.POINTER(ct.c_int), ct.POINTER(SolveInfo)]
    lib.hzs_kappa_gradient.argtypes = [P, P, P, P]
    lib.hzs_precond_get_info.argtypes = [P, ct.POINTER(PrecondInfo)]
    lib.hzs_pipe_peaks.argtypes = [ct.POINTER(PipeRates)]
    lib.hzs_status_string.argtypes = [ct.c_int]
    lib.hzs_status_string.restype = ct.c_char_p
    lib.hzs_last_error.argtypes = [P]
    lib.hzs_last_error.restype = ct.c_char_p
    lib.hzs_version.argtypes = []
    lib.hzs_version.restype = ct.c_char_p
    for name in EXPORTS:
        if name not in ("hzs_grid_destroy", "hzs_precond_destroy", "hzs_status_string", "hzs_last_error",
                        "hzs_version"):
            getattr(lib, name).restype = ct.c_int
    _lib = lib
    return lib


def _check(status: int, grid_ptr=None, allow=(OK,)):
    if status in allow:
        return status
    lib = load()
    msg = lib.hzs_last_error(grid_ptr).decode() or lib.hzs_status_string(status).decode()
    raise HzsError(status, msg)


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ct.c_void_p(s.cuda_stream)


def _dev_c128(t: torch.Tensor, n: int, name: str) -> torch.Tensor:
    if not t.is_cuda or t.dtype != torch.complex128:
        raise TypeError(f"{name} must be a CUDA complex128 tensor")
    if t.shape[-2:] != (n, n) or not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous with trailing shape ({n}, {n})")
    return t


@dataclass
class SolveResult:
    iterations: int
    converged: bool
    relres_est: float
    relres_true: float
    t_solve_ms: float
    t_precond_ms: float
    t_matvec_ms: float
    t_orth_ms: float
    t_orth_dot_ms: float
    t_orth_update_ms: float
    launches: int
    status: int
    basis_bits: int = 0
    orth_kind: int = 0

    @staticmethod
    def of(i) -> "SolveResult":
        return SolveResult(i.iterations, bool(i.converged), i.relres_est, i.relres_true, i.t_solve_ms,
                           i.t_precond_ms, i.t_matvec_ms, i.t_orth_ms, i.t_orth_dot_ms, i.t_orth_update_ms,
                           i.launches, i.status, i.basis_bits, i.orth_kind)


def _solve_flags(profile=False, orth_fp64=False, wide_basis=False, graph=False, basis_df=False,
                 orth_dfma=False) -> int:
    return ((SOLVE_PROFILE if profile else 0) | (SOLVE_ORTH_FP64 if orth_fp64 else 0)
            | (SOLVE_BASIS_WIDE if wide_basis else 0) | (SOLVE_GRAPH if graph else 0)
            | (SOLVE_BASIS_DF if basis_df else 0) | (SOLVE_ORTH_DFMA if orth_dfma else 0))


class Grid:
    """Grid, operator and subdomain decomposition (Sections 2-3)."""

    def __init__(self, n: int, bc: int, k: float = 0.0, kappa: torch.Tensor | None = None,
                 nsub: int = 1, overlap: int = 0, stream=None, nsub_y: int = 0):
        """nsub subdomains along x, nsub_y along y (0: nsub)."""
        lib = load()
        self.n, self.bc, self.k, self.nsub, self.overlap, self.nsub_y = n, bc, k, nsub, overlap, nsub_y
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        kp = None
        if kappa is not None:
            if not kappa.is_cuda or kappa.dtype != torch.float64 or kappa.shape != (n, n):
                raise TypeError("kappa must be a CUDA float64 (n, n) tensor")
            kp = ct.c_void_p(kappa.contiguous().data_ptr())
            self._kappa_ref = kappa
        d = GridDesc(n, bc, float(k), kp, nsub, overlap, nsub_y)
        h = ct.c_void_p()
        _check(lib.hzs_grid_create(ct.byref(d), _stream_ptr(self.stream), ct.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            load().hzs_grid_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Preconditioner:
    """Factorised Schwarz preconditioner (Sections 3-4) on a Grid."""

    def __init__(self, grid: Grid, kind: int = SHS2, coarse: int = COARSE_B2, coarse_ratio: int = 2,
                 precision: int = FP64, dedup_tiles: bool = True, coarse_solver: int = 0, autotune: int = 0,
                 scaling_mode: int = 0, ml: tuple[int, int, int] | None = None):
        """autotune: 0 = default launch shape of the subdomain solve, 1 = pick it by timing at
        set-up (reusing an earlier choice for the same problem size), 2 = always re-time.
        scaling_mode: D_i of SAS2 / SHS2, SCALING_OWNER (0) or SCALING_MULTIPLICITY (1).
        ml: (coarse subdomains per axis, their overlap, coarse-of-coarse ratio) for
        coarse_solver = COARSE_SOLVER_MULTILEVEL."""
        lib = load()
        self.grid = grid
        self.kind, self.coarse, self.coarse_ratio, self.precision = kind, coarse, coarse_ratio, precision
        ml = ml or (0, 0, 0)
        d = PrecondDesc(kind, coarse, coarse_ratio, precision, int(dedup_tiles), int(coarse_solver), int(autotune),
                        int(scaling_mode), int(ml[0]), int(ml[1]), int(ml[2]))
        h = ct.c_void_p()
        _check(lib.hzs_precond_setup(grid.handle, ct.byref(d), ct.byref(h)), grid.handle)
        self._h = h

    @property
    def handle(self):
        return self._h

    @property
    def n(self):
        return self.grid.n

    def apply_operator(self, x: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        x = _dev_c128(x, self.n, "x")
        y = torch.empty_like(x) if out is None else out
        nrhs = x.numel() // (self.n * self.n)
        _check(load().hzs_apply_operator(self._h, x.data_ptr(), y.data_ptr(), nrhs), self.grid.handle)
        return y

    def apply(self, v: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        v = _dev_c128(v, self.n, "v")
        z = torch.empty_like(v) if out is None else out
        nrhs = v.numel() // (self.n * self.n)
        _check(load().hzs_apply_precond(self._h, v.data_ptr(), z.data_ptr(), nrhs), self.grid.handle)
        return z

    def info(self) -> dict:
        """What set-up built and chose (hzs_precond_get_info)."""
        out = PrecondInfo()
        _check(load().hzs_precond_get_info(self._h, ct.byref(out)), self.grid.handle)
        return out.as_dict()

    def _solve(self, fn, f, tol, maxit, out, flags):
        f = _dev_c128(f, self.n, "f")
        u = torch.empty_like(f) if out is None else out
        nrhs = f.numel() // (self.n * self.n)
        infos = (SolveInfo * max(nrhs, 1))()
        sd = SolveDesc(float(tol), int(maxit), flags)
        _check(fn(self._h, ct.byref(sd), f.data_ptr(), u.data_ptr(), nrhs, infos), self.grid.handle,
               allow=(OK, NOT_CONVERGED))
        return u, [SolveResult.of(i) for i in infos[:nrhs]]

    def solve(self, f: torch.Tensor, tol: float = 1e-6, maxit: int = 1000, out=None, profile: bool = False,
              orth_fp64: bool = False, wide_basis: bool = False, graph: bool = False, basis_df: bool = False,
              orth_dfma: bool = False):
        """u = A^{-1} f by preconditioned GMRES; returns (u, [SolveResult per right-hand side]).

        With a MIXED preconditioner the orthogonalisation is the delayed CGS2 on the
        FP64 basis (FP64-accurate reorthogonalisation, the work split between the FP64
        and FP32 pipes) unless
        orth_dfma: the same with every FP64-accurate sum in FP64 FMAs,
        orth_fp64: the classical CGS2 with every product in FP64 (four basis passes a step), or
        basis_df: the delayed CGS2 on the narrower double-float basis, whose remainders are
        bf16 pairs (about 32 bits) for tol >= 1e-7 unless wide_basis (complex64, about 48 bits).
        graph: issue the Arnoldi steps as replayed CUDA graphs of 8 steps each."""
        return self._solve(load().hzs_solve, f, tol, maxit, out,
                           _solve_flags(profile, orth_fp64, wide_basis, graph, basis_df, orth_dfma))

    def adjoint_solve(self, g: torch.Tensor, tol: float = 1e-6, maxit: int = 1000, out=None, profile: bool = False,
                      graph: bool = False):
        """lambda = conj(A)^{-1} g; returns (lambda, results)."""
        return self._solve(load().hzs_adjoint_solve, g, tol, maxit, out, _solve_flags(profile, graph=graph))

    def kappa_gradient(self, u: torch.Tensor, lam: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        u = _dev_c128(u, self.n, "u")
        lam = _dev_c128(lam, self.n, "lam")
        g = torch.empty((self.n, self.n), dtype=torch.float64, device=u.device) if out is None else out
        _check(load().hzs_kappa_gradient(self._h, u.data_ptr(), lam.data_ptr(), g.data_ptr()), self.grid.handle)
        return g

    def close(self):
        if getattr(self, "_h", None):
            load().hzs_precond_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_batched(problems, rhs, tol: float = 1e-6, maxit: int = 1000, orth_fp64: bool = False,
                  wide_basis: bool = False, graph: bool = False, basis_df: bool = False, orth_dfma: bool = False):
    """Batched solve over several problems: ``problems`` is a list of Preconditioner
    handles (distinct), ``rhs`` a matching list of complex128 tensors of shape
    (nrhs_k, n_k, n_k).  Returns (list of solutions, list of lists of SolveResult)."""
    lib = load()
    if len(problems) != len(rhs):
        raise ValueError("one right-hand-side tensor per problem")
    k = len(problems)
    outs = []
    for P, f in zip(problems, rhs):
        _dev_c128(f, P.n, "f")
        outs.append(torch.empty_like(f))
    counts = [f.numel() // (P.n * P.n) for P, f in zip(problems, rhs)]
    total = sum(counts)
    infos = (SolveInfo * max(total, 1))()
    arr = lambda vals: (ct.c_void_p * max(k, 1))(*vals)
    sd = SolveDesc(float(tol), int(maxit),
                   _solve_flags(orth_fp64=orth_fp64, wide_basis=wide_basis, graph=graph, basis_df=basis_df,
                                orth_dfma=orth_dfma))
    st = lib.hzs_solve_batched(k, arr([P.handle.value for P in problems]), ct.byref(sd),
                               arr([f.data_ptr() for f in rhs]), arr([u.data_ptr() for u in outs]),
                               (ct.c_int * max(k, 1))(*counts), infos)
    _check(st, None, allow=(OK, NOT_CONVERGED))
    res, pos = [], 0
    for c in counts:
        res.append([SolveResult.of(i) for i in infos[pos:pos + c]])
        pos += c
    return outs, res


def pipe_peaks() -> dict:
    """Measured arithmetic rates of the current GPU (hzs_pipe_peaks): FP32, packed FP32,
    FP64 in TFLOP/s, integer logic and FP64/FP32 conversions in 10^12 op/s."""
    r = PipeRates()
    _check(load().hzs_pipe_peaks(ct.byref(r)))
    return r.as_dict()


def version() -> str:
    return load().hzs_version().decode()
