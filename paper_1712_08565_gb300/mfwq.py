"""Thin Python binding of libmfwq.so (include/mfwq.h): argument marshalling only.

Every computation runs in the CUDA library; this module checks tensor shapes,
dtypes and devices, passes raw pointers and sizes through ctypes, and turns
status codes into exceptions.  PyTorch provides device memory and streams.
There is no fallback: if the library is missing or no GPU is present the
calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmfwq.so")

MFWQ_OK = 0
STATUS = {0: "MFWQ_OK", -1: "MFWQ_EINVAL", -2: "MFWQ_ENOMEM", -3: "MFWQ_ECUDA", -4: "MFWQ_ESETUP",
          -5: "MFWQ_EBREAKDOWN", -6: "MFWQ_ENOCONV", -7: "MFWQ_ETIMEOUT", -8: "MFWQ_ENAN", -9: "MFWQ_EINTERNAL"}
FD_PRECISION = {"fp64": 0, "tf32": 1, "bf16": 2}
GEOMETRY = {"cube": 0, "ring": 1}
FORCING = {"sines": 0, "ring_exact": 1}
EXACT = {"sines": 0, "ring": 1}

_c_int3 = ctypes.c_int * 3
_c_dptr = ctypes.POINTER(ctypes.c_double)


class SetupDesc(ctypes.Structure):
    _fields_ = [("degree", ctypes.c_int * 3), ("nknots", ctypes.c_int * 3), ("knots", _c_dptr * 3),
                ("mixed", ctypes.c_int), ("fd_precision", ctypes.c_int), ("stream", ctypes.c_void_p)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("maxit", ctypes.c_int), ("inner_rtol", ctypes.c_double),
                ("inner_maxit", ctypes.c_int), ("use_initial_guess", ctypes.c_int), ("force_fp64", ctypes.c_int),
                ("res_hist", _c_dptr), ("fp64_low_fd", ctypes.c_int), ("graph_chunk", ctypes.c_int)]


class ProfileStats(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 24), ("launches", ctypes.c_longlong * 24)]


class SolveInfoC(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iterations", ctypes.c_int), ("outer_iterations", ctypes.c_int),
                ("rel_residual", ctypes.c_double)]


@dataclass
class SolveInfo:
    status: int
    iterations: int
    outer_iterations: int
    rel_residual: float
    history: list | None = None

    @property
    def converged(self) -> bool:
        return self.status == MFWQ_OK


class MfwqError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_LIB = None

# (name, restype, argtypes)
_SIGS = [
    ("mfwq_setup", ctypes.c_int, [ctypes.POINTER(SetupDesc), ctypes.POINTER(ctypes.c_void_p)]),
    ("mfwq_destroy", None, [ctypes.c_void_p]),
    ("mfwq_status_string", ctypes.c_char_p, [ctypes.c_int]),
    ("mfwq_last_error", ctypes.c_char_p, []),
    ("mfwq_sizes", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("mfwq_quad_points", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    ("mfwq_tables_1d", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
     + [ctypes.c_void_p] * 6),
    ("mfwq_eval_coeff", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_void_p]),
    ("mfwq_set_coeff", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("mfwq_eval_mass_coeff", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p]),
    ("mfwq_set_mass_coeff", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double]),
    ("mfwq_grad_mass_coeff", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("mfwq_h1_error", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                     ctypes.POINTER(ctypes.c_double)]),
    ("mfwq_load_vector", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    ("mfwq_apply", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("mfwq_apply_T", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("mfwq_apply_f32", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("fd_precond", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("fd_precond_f32", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("mfwq_solve", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(SolveOpts),
                                  ctypes.POINTER(SolveInfoC)]),
    ("mfwq_solve_T", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(SolveOpts),
                                    ctypes.POINTER(SolveInfoC)]),
    ("mfwq_solve_host", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(SolveOpts),
                                       ctypes.POINTER(SolveInfoC)]),
    ("mfwq_grad_coeff", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("mfwq_sync", ctypes.c_int, [ctypes.c_void_p]),
    ("mfwq_profile_enable", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("mfwq_profile_read", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ProfileStats), ctypes.c_int]),
    ("mfwq_profile_stage_mask", ctypes.c_int, [ctypes.c_void_p, ctypes.c_ulonglong]),
    ("mfwq_stage_name", ctypes.c_char_p, [ctypes.c_int]),
    ("mfwq_kernel_launches", ctypes.c_longlong, []),
    ("mfwq_autotune", ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int)]),
    ("mfwq_set_fp32_path", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("mfwq_set_coeff_field", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                            ctypes.c_double, ctypes.c_int]),
    ("mfwq_fp32_path", ctypes.c_int, [ctypes.c_void_p]),
    ("mfwq_set_fd64_path", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("mfwq_fd64_path", ctypes.c_int, [ctypes.c_void_p]),
    ("mfwq_set_slow_tiling", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    ("mfwq_slow_tiling", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int)]),
    ("mfwq_batch_create", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p)]),
    ("mfwq_batch_destroy", None, [ctypes.c_void_p]),
    ("mfwq_batch_set_grouped", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("mfwq_batch_last_grouped", ctypes.c_int, [ctypes.c_void_p]),
    ("mfwq_batch_solve", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                        ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfoC)]),
    ("mfwq_selftest_bounded_wait", ctypes.c_int, [ctypes.c_longlong, ctypes.c_void_p]),
    ("mfwq_probe_fma_rate", ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    ("mfwq_fd_precond_noalloc", ctypes.c_int, [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_void_p),
                                               ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
]

NOALLOC_MAX_N = 4194304


def fd_precond_noalloc(n, U, UT, lam, r, z, stream=None):
    """mfwq_fd_precond_noalloc: FD preconditioner whose scratch is a fixed
    device array inside the library (no allocation).  n = (n1, n2, n3); U, UT,
    lam: three FP64 CUDA tensors each; r, z: FP64 CUDA tensors of n1 n2 n3
    entries.  Calls whose work overlaps on the GPU must not run concurrently."""
    import torch
    dev = r.device
    nn = (ctypes.c_int * 3)(*[int(v) for v in n])
    N = nn[0] * nn[1] * nn[2]
    Up = (ctypes.c_void_p * 3)(*[_ptr(U[l], torch.float64, nn[l] * nn[l], dev).value for l in range(3)])
    UTp = (ctypes.c_void_p * 3)(*[_ptr(UT[l], torch.float64, nn[l] * nn[l], dev).value for l in range(3)])
    Lp = (ctypes.c_void_p * 3)(*[_ptr(lam[l], torch.float64, nn[l], dev).value for l in range(3)])
    # the library takes its scratch address from the current device, so make
    # r's device current for the call
    with torch.cuda.device(dev):
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        _check(lib().mfwq_fd_precond_noalloc(nn, Up, UTp, Lp, _ptr(r, torch.float64, N, dev),
                                             _ptr(z, torch.float64, N, dev), ctypes.c_void_p(s.cuda_stream)))
    return z


def probe_fma_rate(fp64: bool = True, stream=None) -> float:
    """Measured FMA throughput of the current device in TFLOP/s (mfwq_probe_fma_rate)."""
    v = ctypes.c_double()
    _check(lib().mfwq_probe_fma_rate(1 if fp64 else 0, ctypes.c_void_p(stream.cuda_stream) if stream is not None else None,
                                     ctypes.byref(v)))
    return v.value


def kernel_launches() -> int:
    """Kernels the library has launched in this process (all handles)."""
    return int(lib().mfwq_kernel_launches())


def lib():
    """Load libmfwq.so (built in-tree by paper_1712_08565_gb300.build)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1712_08565_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in _SIGS:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def _check(st: int):
    if st != MFWQ_OK:
        msg = lib().mfwq_last_error().decode() or lib().mfwq_status_string(st).decode()
        raise MfwqError(st, msg)


def tables_1d(degree: int, knots) -> dict:
    """Host-only 1D tables of the library (no GPU needed): points, B0, B1,
    the four weight families (index 2a+b), FD eigenvectors and eigenvalues."""
    k = np.ascontiguousarray(knots, dtype=np.float64)
    n, nq = ctypes.c_int(), ctypes.c_int()
    _check(lib().mfwq_tables_1d(degree, len(k), k.ctypes.data, ctypes.byref(n), ctypes.byref(nq),
                                None, None, None, None, None, None))
    n, nq = n.value, nq.value
    out = dict(xq=np.zeros(nq), B0=np.zeros((nq, n)), B1=np.zeros((nq, n)), W=np.zeros((4, n, nq)),
               U=np.zeros((n, n)), lam=np.zeros(n))
    _check(lib().mfwq_tables_1d(degree, len(k), k.ctypes.data, ctypes.byref(ctypes.c_int()), ctypes.byref(ctypes.c_int()),
                                *(out[x].ctypes.data for x in ("xq", "B0", "B1", "W", "U", "lam"))))
    return out


def _ptr(t, dtype, numel=None, device=None):
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch.Tensor")
    if t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    if not t.is_cuda:
        raise ValueError("tensor must be on a CUDA device")
    if device is not None and t.device != device:
        raise ValueError(f"tensor on {t.device}, operator on {device}")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"expected {numel} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


class Operator:
    """One MF-WQ patch: tables, coefficient and workspace on one GPU.

    degree: int or 3 ints; knots: 3 open knot vectors (direction 1, 2, 3).
    mixed: also build the FP32 operator and tensor-core FD for the
    mixed-precision solve; fd_precision: 'tf32' or 'bf16'.
    """

    def __init__(self, degree, knots, mixed: bool = False, fd_precision: str = "tf32", device=None, stream=None):
        import torch
        if device is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        else:
            self.device = torch.device(device)
            if self.device.index is None:
                self.device = torch.device("cuda", torch.cuda.current_device())
        degs = [int(degree)] * 3 if np.ndim(degree) == 0 else [int(d) for d in degree]
        self._knots = [np.ascontiguousarray(k, dtype=np.float64) for k in knots]
        desc = SetupDesc()
        for l in range(3):
            desc.degree[l] = degs[l]
            desc.nknots[l] = len(self._knots[l])
            desc.knots[l] = self._knots[l].ctypes.data_as(_c_dptr)
        desc.mixed = 1 if mixed else 0
        desc.fd_precision = FD_PRECISION[fd_precision] if mixed else 0
        with torch.cuda.device(self.device):
            s = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.stream = s
            desc.stream = ctypes.c_void_p(s.cuda_stream)
            h = ctypes.c_void_p()
            _check(lib().mfwq_setup(ctypes.byref(desc), ctypes.byref(h)))
        self._h = h
        self.degree = degs
        self.mixed = bool(mixed)
        self.fd_precision = fd_precision if mixed else "fp64"
        n, nq = _c_int3(), _c_int3()
        _check(lib().mfwq_sizes(self._h, n, nq))
        self.n = tuple(n)
        self.nq = tuple(nq)
        self.shape = (self.n[2], self.n[1], self.n[0])
        self.qshape = (self.nq[2], self.nq[1], self.nq[0])
        self.N = self.n[0] * self.n[1] * self.n[2]
        self.Nq = self.nq[0] * self.nq[1] * self.nq[2]

    # ------------------------------------------------------------ lifetime
    def close(self):
        if getattr(self, "_h", None):
            lib().mfwq_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ helpers
    def _new(self, shape, dtype):
        import torch
        return torch.empty(shape, dtype=dtype, device=self.device)

    def quad_points(self, direction: int) -> np.ndarray:
        out = np.zeros(self.nq[direction])
        _check(lib().mfwq_quad_points(self._h, direction, out.ctypes.data))
        return out

    # ------------------------------------------------------------ setup helpers
    def eval_coeff(self, geometry: str = "ring", modes=None, kscale: float = 0.0, out=None):
        import torch
        out = out if out is not None else self._new((6,) + self.qshape, torch.float64)
        m = np.ascontiguousarray(modes if modes is not None else np.zeros((0, 5)), dtype=np.float64)
        _check(lib().mfwq_eval_coeff(self._h, GEOMETRY[geometry], m.ctypes.data if m.size else None, int(m.shape[0]),
                                     float(kscale), _ptr(out, torch.float64, 6 * self.Nq, self.device)))
        return out

    def set_coeff_field(self, geometry: str = "ring", modes=None, kscale: float = 0.0, onthefly: bool = True):
        """Coefficient from its definition (mfwq_set_coeff_field): the FP64
        fields stored; with onthefly the FP32 operator evaluates C in its x
        stage instead of storing an FP32 copy."""
        m = np.ascontiguousarray(modes if modes is not None else np.zeros((0, 5)), dtype=np.float64)
        _check(lib().mfwq_set_coeff_field(self._h, GEOMETRY[geometry], m.ctypes.data if m.size else None,
                                          int(m.shape[0]), float(kscale), 1 if onthefly else 0))

    def set_coeff(self, C):
        import torch
        _check(lib().mfwq_set_coeff(self._h, _ptr(C, torch.float64, 6 * self.Nq, self.device)))

    def eval_mass_coeff(self, geometry: str = "ring", alpha: float = 1.0, out=None):
        """c = alpha |det J| at the WQ points, shape (nq3, nq2, nq1) (mfwq_eval_mass_coeff)."""
        import torch
        out = out if out is not None else self._new(self.qshape, torch.float64)
        _check(lib().mfwq_eval_mass_coeff(self._h, GEOMETRY[geometry], float(alpha),
                                          _ptr(out, torch.float64, self.Nq, self.device)))
        return out

    def set_mass_coeff(self, c=None, fd_shift: float = 0.0):
        """Turn the reaction term on with c at the WQ points (None: off) and set
        the FD shift (mfwq_set_mass_coeff)."""
        import torch
        ptr = None if c is None else _ptr(c, torch.float64, self.Nq, self.device)
        _check(lib().mfwq_set_mass_coeff(self._h, ptr, float(fd_shift)))

    def grad_mass_coeff(self, lam, u, out=None):
        """dJ/dc at the WQ points (mfwq_grad_mass_coeff)."""
        import torch
        out = out if out is not None else self._new(self.qshape, torch.float64)
        _check(lib().mfwq_grad_mass_coeff(self._h, _ptr(lam, torch.float64, self.N, self.device),
                                          _ptr(u, torch.float64, self.N, self.device),
                                          _ptr(out, torch.float64, self.Nq, self.device)))
        return out

    def h1_error(self, u, geometry: str = "ring", solution: str = "ring") -> float:
        """Relative H1 error of the discrete function u against an exact
        solution ('sines' on the cube, 'ring' = Eq. (exact-solution)); synchronous."""
        import torch
        v = ctypes.c_double()
        _check(lib().mfwq_h1_error(self._h, GEOMETRY[geometry], EXACT[solution],
                                   _ptr(u, torch.float64, self.N, self.device), ctypes.byref(v)))
        return v.value

    def load_vector(self, geometry: str = "ring", forcing: str = "sines", out=None):
        import torch
        out = out if out is not None else self._new(self.shape, torch.float64)
        _check(lib().mfwq_load_vector(self._h, GEOMETRY[geometry], FORCING[forcing], _ptr(out, torch.float64, self.N, self.device)))
        return out

    # ------------------------------------------------------------ hot path
    def apply(self, x, out=None):
        import torch
        out = out if out is not None else self._new(self.shape, torch.float64)
        _check(lib().mfwq_apply(self._h, _ptr(x, torch.float64, self.N, self.device), _ptr(out, torch.float64, self.N, self.device)))
        return out

    def apply_T(self, x, out=None):
        import torch
        out = out if out is not None else self._new(self.shape, torch.float64)
        _check(lib().mfwq_apply_T(self._h, _ptr(x, torch.float64, self.N, self.device), _ptr(out, torch.float64, self.N, self.device)))
        return out

    def apply_f32(self, x, out=None):
        import torch
        out = out if out is not None else self._new(self.shape, torch.float32)
        _check(lib().mfwq_apply_f32(self._h, _ptr(x, torch.float32, self.N, self.device), _ptr(out, torch.float32, self.N, self.device)))
        return out

    def fd_precond(self, r, out=None):
        import torch
        out = out if out is not None else self._new(self.shape, torch.float64)
        _check(lib().fd_precond(self._h, _ptr(r, torch.float64, self.N, self.device), _ptr(out, torch.float64, self.N, self.device)))
        return out

    def fd_precond_f32(self, r, out=None):
        import torch
        out = out if out is not None else self._new(self.shape, torch.float32)
        _check(lib().fd_precond_f32(self._h, _ptr(r, torch.float32, self.N, self.device), _ptr(out, torch.float32, self.N, self.device)))
        return out

    def _opts(self, rtol, maxit, inner_rtol, inner_maxit, x0, force_fp64, history, fp64_low_fd=False, graph_chunk=0):
        o = SolveOpts()
        o.fp64_low_fd = 1 if fp64_low_fd else 0
        o.graph_chunk = int(graph_chunk)
        o.rtol = rtol
        o.maxit = maxit
        o.inner_rtol = inner_rtol
        o.inner_maxit = inner_maxit
        o.use_initial_guess = 1 if x0 else 0
        o.force_fp64 = 1 if force_fp64 else 0
        hist = None
        if history:
            hist = np.zeros(maxit + 2)
            o.res_hist = hist.ctypes.data_as(_c_dptr)
        return o, hist

    def _solve(self, fn, f, u, rtol, maxit, inner_rtol, inner_maxit, force_fp64, history, check, fp64_low_fd=False,
               graph_chunk=0):
        import torch
        x0 = u is not None
        u = u if u is not None else self._new(self.shape, torch.float64)
        o, hist = self._opts(rtol, maxit, inner_rtol, inner_maxit, x0, force_fp64, history, fp64_low_fd, graph_chunk)
        info = SolveInfoC()
        st = fn(self._h, _ptr(f, torch.float64, self.N, self.device), _ptr(u, torch.float64, self.N, self.device),
                ctypes.byref(o), ctypes.byref(info))
        if st not in (MFWQ_OK, -6, -5, -8) or (check and st != MFWQ_OK):
            _check(st)
        h = None
        if hist is not None:
            last = info.outer_iterations if (self.mixed and not force_fp64 and not fp64_low_fd) else info.iterations
            h = list(hist[: last + 1])
        return u, SolveInfo(info.status, info.iterations, info.outer_iterations, info.rel_residual, h)

    def solve(self, f, u=None, rtol=1e-10, maxit=500, inner_rtol=0.0, inner_maxit=0, force_fp64=False,
              history=False, check=False, fp64_low_fd=False, graph_chunk=0):
        """Solve K~ u = f (FP64 BiCGStab + FD, or mixed refinement on a mixed
        operator).  u, if given, is the initial guess and receives the result.
        fp64_low_fd (mixed operator): FP64 BiCGStab with the FD in the
        operator's low precision (tensor cores); the tolerance is met in FP64.
        graph_chunk > 1: FP64 iterations captured that many to a CUDA graph
        (needs an operator on a non-default stream)."""
        return self._solve(lib().mfwq_solve, f, u, rtol, maxit, inner_rtol, inner_maxit, force_fp64, history, check,
                           fp64_low_fd, graph_chunk)

    def solve_T(self, g, lam=None, rtol=1e-10, maxit=500, history=False, check=False, fp64_low_fd=False):
        """Solve the adjoint system K~^T lambda = g (FP64; fp64_low_fd as in solve)."""
        return self._solve(lib().mfwq_solve_T, g, lam, rtol, maxit, 0.0, 0, True, history, check, fp64_low_fd)

    def solve_host(self, f_host: np.ndarray, out: np.ndarray | None = None, x0: np.ndarray | None = None,
                   rtol=1e-10, maxit=500, inner_rtol=0.0, inner_maxit=0, force_fp64=False):
        """mfwq_solve with host arrays (copies inside the call).  out receives
        u; x0, if given, is the initial guess."""
        f = np.ascontiguousarray(f_host, dtype=np.float64)
        u = out if out is not None else np.empty(self.shape)
        if not (u.flags.c_contiguous and u.dtype == np.float64 and u.size == self.N):
            raise ValueError("out must be a C-contiguous float64 array of N entries")
        if x0 is not None:
            u[...] = np.asarray(x0, dtype=np.float64).reshape(u.shape)
        o, _ = self._opts(rtol, maxit, inner_rtol, inner_maxit, x0 is not None, force_fp64, False)
        info = SolveInfoC()
        st = lib().mfwq_solve_host(self._h, f.ctypes.data, u.ctypes.data, ctypes.byref(o), ctypes.byref(info))
        if st not in (MFWQ_OK, -6):
            _check(st)
        return u, SolveInfo(info.status, info.iterations, info.outer_iterations, info.rel_residual)

    def grad_coeff(self, lam, u, out=None):
        import torch
        out = out if out is not None else self._new((6,) + self.qshape, torch.float64)
        _check(lib().mfwq_grad_coeff(self._h, _ptr(lam, torch.float64, self.N, self.device), _ptr(u, torch.float64, self.N, self.device),
                                     _ptr(out, torch.float64, 6 * self.Nq, self.device)))
        return out

    def sync(self):
        _check(lib().mfwq_sync(self._h))

    def autotune(self, cache_path: str | None = None) -> int:
        """Pick the apply's launch shapes by timing (mfwq_autotune); returns the
        FP64 choice as 1000 * reduced carveout + 100 * slow-stage rows
        + 10 * x-stage mapping + lines."""
        v = ctypes.c_int()
        _check(lib().mfwq_autotune(self._h, cache_path.encode() if cache_path else None, ctypes.byref(v)))
        return v.value

    @property
    def fp32_path(self) -> str:
        """Kernel sequence of the FP32 operator: 'staged' or 'fused' (mfwq_fp32_path)."""
        v = lib().mfwq_fp32_path(self._h)
        if v < 0:
            _check(v)
        return "fused" if v == 1 else "staged"

    @fp32_path.setter
    def fp32_path(self, path: str):
        _check(lib().mfwq_set_fp32_path(self._h, {"staged": 0, "fused": 1}[path]))

    @property
    def fd64_path(self) -> str:
        """Kernels of the FP64 FD: 'pipe' (FP64 pipe) or 'split' (BF16 tensor
        cores by operand splitting), mfwq_fd64_path."""
        v = lib().mfwq_fd64_path(self._h)
        if v < 0:
            _check(v)
        return "split" if v == 1 else "pipe"

    @fd64_path.setter
    def fd64_path(self, path: str):
        _check(lib().mfwq_set_fd64_path(self._h, {"pipe": 0, "split": 1}[path]))

    def slow_tiling(self, fp32: bool = False) -> tuple[int, int]:
        """(rows, cols) per thread of the slow-dimension stages (mfwq_slow_tiling)."""
        r, c = ctypes.c_int(), ctypes.c_int()
        _check(lib().mfwq_slow_tiling(self._h, 1 if fp32 else 0, ctypes.byref(r), ctypes.byref(c)))
        return r.value, c.value

    def set_slow_tiling(self, rows: int, cols: int = 1, fp32: bool = False):
        """Thread tiling of the slow-dimension stages (mfwq_set_slow_tiling)."""
        _check(lib().mfwq_set_slow_tiling(self._h, 1 if fp32 else 0, rows, cols))

    def profile(self, on: bool = True):
        """Bracket every later kernel launch with CUDA events (per-stage timing)."""
        _check(lib().mfwq_profile_enable(self._h, 1 if on else 0))

    def profile_stages(self, names=None):
        """Bracket only the named stages with events while profiling (None: all)."""
        mask = (1 << 64) - 1
        if names is not None:
            idx = {lib().mfwq_stage_name(i).decode(): i for i in range(24)}
            mask = 0
            for n in names:
                mask |= 1 << idx[n]
        _check(lib().mfwq_profile_stage_mask(self._h, ctypes.c_ulonglong(mask)))

    def profile_read(self, reset: bool = True) -> dict:
        """{stage name: (device ms summed, launches)} since the last reset."""
        st = ProfileStats()
        _check(lib().mfwq_profile_read(self._h, ctypes.byref(st), 1 if reset else 0))
        out = {}
        for i in range(24):
            if st.launches[i]:
                out[lib().mfwq_stage_name(i).decode()] = (st.ms[i], int(st.launches[i]))
        return out


def _make_solve_function():
    import torch

    class MfwqSolve(torch.autograd.Function):
        """u = K~(C)^-1 f with gradients for C (6 symmetric fields at the WQ
        points) and f.  Backward solves the adjoint K~^T lambda = dL/du and
        returns dL/dC = -fold((W^T lambda) (B u)) and dL/df = lambda."""

        @staticmethod
        def forward(ctx, C6, f, op: Operator, rtol: float):
            op.set_coeff(C6.contiguous())
            u, info = op.solve(f.contiguous(), rtol=rtol, force_fp64=True)
            if not info.converged:
                raise MfwqError(info.status, "forward solve did not converge")
            ctx.op = op
            ctx.rtol = rtol
            ctx.save_for_backward(C6, u)
            return u

        @staticmethod
        def backward(ctx, grad_u):
            C6, u = ctx.saved_tensors
            op = ctx.op
            op.set_coeff(C6.contiguous())
            lam, info = op.solve_T(grad_u.contiguous(), rtol=ctx.rtol)
            if not info.converged:
                raise MfwqError(info.status, "adjoint solve did not converge")
            gC = op.grad_coeff(lam, u)
            return gC, lam, None, None

    return MfwqSolve


_SOLVE_FN = None


def solve_fn():
    """torch.autograd.Function applying u = K~(C)^-1 f: solve_fn().apply(C6, f, op, rtol)."""
    global _SOLVE_FN
    if _SOLVE_FN is None:
        _SOLVE_FN = _make_solve_function()
    return _SOLVE_FN


class Batch:
    """Independent patches solved together (mfwq_batch_*): one CUDA graph
    launch per BiCGStab sweep over all patches.  The operators stay owned by
    the caller and must outlive the batch."""

    def __init__(self, ops):
        self.ops = list(ops)
        arr = (ctypes.c_void_p * len(self.ops))(*[op._h.value for op in self.ops])
        h = ctypes.c_void_p()
        _check(lib().mfwq_batch_create(len(self.ops), arr, ctypes.byref(h)))
        self._h = h

    @property
    def grouped(self) -> bool:
        """True if the last FP64 solve ran grouped sweeps (mfwq_batch_last_grouped)."""
        return bool(lib().mfwq_batch_last_grouped(self._h))

    def set_grouped(self, groups: int):
        """FP64 sweeps as grouped launches in `groups` concurrent groups of
        patches (0: per-patch streams, the default) (mfwq_batch_set_grouped)."""
        _check(lib().mfwq_batch_set_grouped(self._h, int(groups)))

    def close(self):
        if getattr(self, "_h", None):
            lib().mfwq_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, fs, us=None, rtol=1e-8, maxit=500, force_fp64=False, inner_rtol=0.0, inner_maxit=0, x0=False,
              check=False):
        """Solve every patch; FP64 (force_fp64 or any non-mixed patch) or the
        mixed refinement (all patches mixed).  With x0, us holds the initial guesses."""
        import torch
        n = len(self.ops)
        us = us if us is not None else [torch.empty_like(f) for f in fs]
        fp = (ctypes.c_void_p * n)(*[_ptr(fs[i], torch.float64, self.ops[i].N, self.ops[i].device).value for i in range(n)])
        up = (ctypes.c_void_p * n)(*[_ptr(us[i], torch.float64, self.ops[i].N, self.ops[i].device).value for i in range(n)])
        o = SolveOpts()
        o.rtol = rtol
        o.maxit = maxit
        o.force_fp64 = 1 if force_fp64 else 0
        o.inner_rtol = inner_rtol
        o.inner_maxit = inner_maxit
        o.use_initial_guess = 1 if x0 else 0
        infos = (SolveInfoC * n)()
        st = lib().mfwq_batch_solve(self._h, fp, up, ctypes.byref(o), infos)
        if st not in (MFWQ_OK, -6, -5, -8) or (check and st != MFWQ_OK):
            _check(st)
        return us, [SolveInfo(x.status, x.iterations, x.outer_iterations, x.rel_residual) for x in infos]
