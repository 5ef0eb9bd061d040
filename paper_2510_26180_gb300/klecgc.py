"""ctypes binding of include/klecgc.h (same names, argument marshalling only).

Arrays may be torch tensors (CUDA or CPU) or numpy arrays; they are passed
to the library as raw pointers, and the library decides host/device from the
pointer.  The CUDA stream defaults to torch's current stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

FP64, MIXED, MIXED_DEFECT = 0, 1, 2
GUESS_GPC, GUESS_ZERO, GUESS_USER, GUESS_COARSE, GUESS_MLP = 0, 1, 2, 3, 4
(OK, E_INVALID_ARG, E_OUT_OF_MEMORY, E_NOT_CONVERGED, E_NONFINITE, E_CUDA,
 E_UNSUPPORTED) = range(7)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libklecgc.so")

# Every symbol declared in include/klecgc.h.
EXPORTS = ["klecgc_setup", "klecgc_solve", "klecgc_field", "klecgc_guess", "klecgc_fine_sweep",
           "klecgc_cgc_apply", "klecgc_reference", "klecgc_info", "klecgc_free",
           "klecgc_status_string", "klecgc_last_error", "klecgc_profile_enable",
           "klecgc_profile_read", "klecgc_reference_noalloc", "klecgc_mlp_set", "klecgc_mlp_get",
           "klecgc_mlp_loss_grad", "klecgc_mlp_train", "klecgc_mlp_guess", "klecgc_downsample",
           "klecgc_mlp_set_residual", "klecgc_mlp_targets",
           "klecgc_set_krylov", "klecgc_set_2d_method", "klecgc_set_loop",
           "klecgc_set_tuning", "klecgc_tuning_report",
           "klecgc_set_scratch_limit",
           "klecgc_krylov_stats", "klecgc_save", "klecgc_load",
           "klecgc_solve_batch", "klecgc_solve_parareal", "klecgc_kl_basis",
           "klecgc_gpc_indices"]
PROFILE_CLASSES = ["field", "factors", "guess", "fine", "cgc_fwd", "cgc_solve", "cgc_inv",
                   "conv", "layout"]


class KlecgcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"klecgc status {status}: {msg}")
        self.status = status


class Problem(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("nx", ctypes.c_int32), ("T", ctypes.c_double),
                ("sigma", ctypes.c_double), ("corr_len", ctypes.c_double),
                ("M", ctypes.c_int32), ("gpc_degree", ctypes.c_int32),
                ("n_train", ctypes.c_int32), ("eps_kl", ctypes.c_double),
                ("N", ctypes.c_int32), ("J", ctypes.c_int32), ("reaction", ctypes.c_double),
                ("forcing", ctypes.c_double), ("u0_kind", ctypes.c_int32),
                ("reaction_kind", ctypes.c_int32), ("cgc_newton", ctypes.c_int32),
                ("advection", ctypes.c_double)]

    @classmethod
    def from_workload(cls, w) -> "Problem":
        return cls(dim=w.dim, nx=w.nx, T=w.T, sigma=w.sigma, corr_len=w.corr_len, M=w.M,
                   gpc_degree=w.gpc_degree, n_train=w.n_train, eps_kl=w.eps_kl, N=w.N, J=w.J,
                   reaction=w.reaction, forcing=w.forcing, u0_kind=w.u0_kind,
                   reaction_kind=getattr(w, "reaction_kind", 0),
                   cgc_newton=getattr(w, "cgc_newton", 1),
                   advection=getattr(w, "advection", 0.0))


class Instance(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_int32), ("J", ctypes.c_int32)]


class Profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64 * 16), ("ms", ctypes.c_double * 16),
                ("n_classes", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("N", ctypes.c_int32), ("J", ctypes.c_int32),
                ("M", ctypes.c_int32), ("P", ctypes.c_int32), ("MQ", ctypes.c_int32),
                ("lambda_sum", ctypes.c_double), ("lambda_kept", ctypes.c_double),
                ("n_unknowns", ctypes.c_int32), ("device", ctypes.c_int32)]


_lib = None


def load() -> ctypes.CDLL:
    """Loads the compiled library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    P, D, I64, I32 = ctypes.c_void_p, ctypes.c_double, ctypes.c_int64, ctypes.c_int32
    sig = {
        "klecgc_setup": [ctypes.POINTER(Problem), P, ctypes.POINTER(P), P],
        "klecgc_solve": [P, P, I64, D, I32, I32, D, D, I32, I32, I32, P, P, P, P, P],
        "klecgc_field": [P, P, I64, P, P],
        "klecgc_guess": [P, P, I64, I32, P, P],
        "klecgc_fine_sweep": [P, P, I64, I32, P, D, I32, D, I32, P, P],
        "klecgc_cgc_apply": [P, P, I64, I32, P, D, D, I32, P, P],
        "klecgc_reference": [P, P, I64, I32, I32, P, P],
        "klecgc_reference_noalloc": [P, P, I64, I32, I32, P, P],
        "klecgc_info": [P, ctypes.POINTER(Info)],
        "klecgc_profile_enable": [P, I32],
        "klecgc_mlp_set": [P, P, I64, P, P],
        "klecgc_mlp_get": [P, P, P, P, ctypes.POINTER(ctypes.c_int64)],
        "klecgc_mlp_loss_grad": [P, P, P, I64, ctypes.POINTER(ctypes.c_double), P, P],
        "klecgc_mlp_train": [P, P, P, I64, I32, I32, D, D, ctypes.c_uint64, I32, P, P],
        "klecgc_mlp_guess": [P, P, I64, P, P],
        "klecgc_downsample": [P, P, I64, I32, P, P],
        "klecgc_mlp_set_residual": [P, I32],
        "klecgc_mlp_targets": [P, P, P, I64, P, P],
        "klecgc_profile_read": [P, ctypes.POINTER(Profile)],
        "klecgc_set_krylov": [P, D, D, I32],
        "klecgc_set_2d_method": [P, I32],
        "klecgc_set_loop": [P, I32],
        "klecgc_set_tuning": [P, I32, ctypes.c_char_p],
        "klecgc_tuning_report": [P, ctypes.c_char_p, I64, P],
        "klecgc_set_scratch_limit": [P, I64],
        "klecgc_solve_parareal": [P, P, I64, D, I32, I32, D, I32, I32, P, P, P, P, P],
        "klecgc_save": [P, ctypes.c_char_p],
        "klecgc_load": [ctypes.c_char_p, ctypes.POINTER(P), P],
        "klecgc_solve_batch": [ctypes.POINTER(P), I32, ctypes.POINTER(Instance), I64, P, D, D,
                               I32, I32, I32, P, P, P, P],
        "klecgc_krylov_stats": [P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)],
        "klecgc_kl_basis": [I32, D, D, I32, P, I64, P, P],
        "klecgc_gpc_indices": [I32, I32, P, I64, ctypes.POINTER(ctypes.c_int64)],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.klecgc_free.argtypes = [P]
    lib.klecgc_free.restype = None
    lib.klecgc_status_string.argtypes = [ctypes.c_int]
    lib.klecgc_status_string.restype = ctypes.c_char_p
    lib.klecgc_last_error.argtypes = []
    lib.klecgc_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def exported_symbols():
    """Names of EXPORTS that the loaded library actually exports."""
    lib = load()
    return [n for n in EXPORTS if hasattr(lib, n)]


def _ptr(a, dtype):
    """Raw pointer of a contiguous torch tensor / numpy array of `dtype`."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
            raise TypeError(f"expected a C-contiguous {dtype} array")
        return a.ctypes.data
    import torch
    tdt = {np.float64: torch.float64, np.int32: torch.int32, np.float32: torch.float32}[dtype]
    if a.dtype != tdt or not a.is_contiguous():
        raise TypeError(f"expected a contiguous {tdt} tensor")
    return a.data_ptr()


def _stream(stream):
    if stream is not None:
        return getattr(stream, "cuda_stream", stream)
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return None


def _check(status: int, allow=(OK,)) -> int:
    if status not in allow:
        lib = load()
        raise KlecgcError(status, lib.klecgc_last_error().decode())
    return status


def solve_batch(solvers, ctx_index, J, xi, alpha, tol, kmax, precision, guess, U_out,
                iters_out=None, status_out=None, stream=None,
                allow=(OK, E_NOT_CONVERGED, E_NONFINITE)) -> int:
    """klecgc_solve_batch: instance i uses solvers[ctx_index[i]] and J[i] fine
    steps; U_out is the packed per-instance output (see the header)."""
    lib = load()
    n = len(ctx_index)
    inst = (Instance * max(n, 1))()
    for i in range(n):
        inst[i].ctx = int(ctx_index[i])
        inst[i].J = int(J[i])
    handles = (ctypes.c_void_p * len(solvers))(*[s.h.value for s in solvers])
    return _check(lib.klecgc_solve_batch(handles, len(solvers), inst, n, _ptr(xi, np.float64),
                                         alpha, tol, kmax, precision, guess,
                                         _ptr(U_out, np.float64), _ptr(iters_out, np.int32),
                                         _ptr(status_out, np.int32), _stream(stream)), allow)


def kl_basis(dim, corr_len, sigma, M, x):
    """klecgc_kl_basis: the input-KL basis sqrt(lambda_m) phi_m at the points
    x ([n] in 1D, [n][2] in 2D); returns (basis [M][n], lambda [M])."""
    lib = load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.shape[0] if x.ndim else 0
    out = np.empty((M, n))
    lam = np.empty(M)
    _check(lib.klecgc_kl_basis(dim, corr_len, sigma, M, _ptr(x, np.float64), n,
                               _ptr(out, np.float64), _ptr(lam, np.float64)))
    return out, lam


def gpc_indices(M, p):
    """klecgc_gpc_indices: the gPC multi-indices [P][M] in the library's order."""
    lib = load()
    P = ctypes.c_int64()
    _check(lib.klecgc_gpc_indices(M, p, None, 0, ctypes.byref(P)))
    out = np.empty((P.value, M), dtype=np.int32)
    _check(lib.klecgc_gpc_indices(M, p, _ptr(out, np.int32), P.value, ctypes.byref(P)))
    return out

class Solver:
    """Owns one klecgc context (klecgc_setup ... klecgc_free)."""

    def __init__(self, problem: Problem, xi_train, stream=None):
        self.lib = load()
        self.problem = problem
        h = ctypes.c_void_p()
        _check(self.lib.klecgc_setup(ctypes.byref(problem), _ptr(xi_train, np.float64),
                                     ctypes.byref(h), _stream(stream)))
        self.h = h

    @classmethod
    def load(cls, path: str, stream=None) -> "Solver":
        """A solver from a context file written by save()."""
        self = cls.__new__(cls)
        self.lib = load()
        self.problem = None
        h = ctypes.c_void_p()
        _check(self.lib.klecgc_load(os.fsencode(path), ctypes.byref(h), _stream(stream)))
        self.h = h
        return self

    def save(self, path: str) -> int:
        return _check(self.lib.klecgc_save(self.h, os.fsencode(path)))

    def close(self):
        if getattr(self, "h", None):
            self.lib.klecgc_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> Info:
        out = Info()
        _check(self.lib.klecgc_info(self.h, ctypes.byref(out)))
        return out

    def profile_enable(self, timing: bool) -> None:
        _check(self.lib.klecgc_profile_enable(self.h, 1 if timing else 0))

    def profile_read(self) -> dict:
        """{class: (launches, summed ms)} since the last profile_enable."""
        p = Profile()
        _check(self.lib.klecgc_profile_read(self.h, ctypes.byref(p)))
        return {n: (int(p.launches[i]), float(p.ms[i])) for i, n in enumerate(PROFILE_CLASSES)}

    def solve(self, xi, S, dT, J, N, alpha, tol, kmax, precision, guess, U_out,
              iters_out=None, status_out=None, U_guess=None, stream=None,
              allow=(OK, E_NOT_CONVERGED, E_NONFINITE)) -> int:
        return _check(self.lib.klecgc_solve(
            self.h, _ptr(xi, np.float64), S, dT, J, N, alpha, tol, kmax, precision, guess,
            _ptr(U_guess, np.float64), _ptr(U_out, np.float64), _ptr(iters_out, np.int32),
            _ptr(status_out, np.int32), _stream(stream)), allow)

    def solve_parareal(self, xi, S, dT, J, N, tol, kmax, guess, U_out, iters_out=None,
                       status_out=None, U_guess=None, stream=None,
                       allow=(OK, E_NOT_CONVERGED, E_NONFINITE)) -> int:
        """Classical parareal (Algorithm 1): the paper's comparison method."""
        return _check(self.lib.klecgc_solve_parareal(
            self.h, _ptr(xi, np.float64), S, dT, J, N, tol, kmax, guess,
            _ptr(U_guess, np.float64), _ptr(U_out, np.float64), _ptr(iters_out, np.int32),
            _ptr(status_out, np.int32), _stream(stream)), allow)

    def field(self, xi, S, a_out, stream=None) -> int:
        return _check(self.lib.klecgc_field(self.h, _ptr(xi, np.float64), S,
                                            _ptr(a_out, np.float64), _stream(stream)))

    def guess(self, xi, S, precision, U0_out, stream=None) -> int:
        return _check(self.lib.klecgc_guess(self.h, _ptr(xi, np.float64), S, precision,
                                            _ptr(U0_out, np.float64), _stream(stream)))

    def fine_sweep(self, xi, S, N, U_in, dT, J, alpha, precision, r_out, stream=None) -> int:
        return _check(self.lib.klecgc_fine_sweep(
            self.h, _ptr(xi, np.float64), S, N, _ptr(U_in, np.float64), dT, J, alpha, precision,
            _ptr(r_out, np.float64), _stream(stream)))

    def cgc_apply(self, xi, S, N, r_in, dT, alpha, precision, u_out, stream=None) -> int:
        return _check(self.lib.klecgc_cgc_apply(
            self.h, _ptr(xi, np.float64), S, N, _ptr(r_in, np.float64), dT, alpha, precision,
            _ptr(u_out, np.float64), _stream(stream)))

    def reference(self, xi, S, N, J, U_out, stream=None) -> int:
        return _check(self.lib.klecgc_reference(self.h, _ptr(xi, np.float64), S, N, J,
                                                 _ptr(U_out, np.float64), _stream(stream)))

    # ---- 2D Krylov solves
    def set_krylov(self, rtol_fine, rtol_cgc, maxit) -> int:
        return _check(self.lib.klecgc_set_krylov(self.h, rtol_fine, rtol_cgc, maxit))

    def set_scratch_limit(self, nbytes) -> int:
        """Budget for the context's device scratch in bytes (0: none)."""
        return _check(self.lib.klecgc_set_scratch_limit(self.h, int(nbytes)))

    def set_tuning(self, mode, cache_path=None) -> int:
        """Launch-shape autotuner: 1 time the candidates once per shape, 0 fixed rules."""
        path = cache_path.encode() if cache_path else None
        return _check(self.lib.klecgc_set_tuning(self.h, mode, path))

    def tuning_report(self) -> dict:
        """The autotuner's choices, {key: shape}."""
        import json
        n = ctypes.c_int64(0)
        _check(self.lib.klecgc_tuning_report(self.h, None, 0, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value + 1)
        _check(self.lib.klecgc_tuning_report(self.h, buf, n.value + 1, ctypes.byref(n)))
        return json.loads(buf.value.decode())

    def set_loop(self, mode) -> int:
        """Parareal loop: 0 CUDA graph with a WHILE node (default), 1 host-driven."""
        return _check(self.lib.klecgc_set_loop(self.h, mode))

    def set_2d_method(self, method) -> int:
        """0 auto (banded LU in FP64 for nx <= 32), 1 Krylov, 2 banded LU (nx <= 64),
        3 Krylov with the mixed fine systems on thread-block clusters."""
        return _check(self.lib.klecgc_set_2d_method(self.h, method))

    def krylov_stats(self) -> tuple:
        """(fine, CGC) Krylov iterations summed over the systems of the last call."""
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check(self.lib.klecgc_krylov_stats(self.h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    # ---- learned guess
    def mlp_n_params(self) -> int:
        n = ctypes.c_int64()
        _check(self.lib.klecgc_mlp_get(self.h, None, None, None, ctypes.byref(n)))
        return n.value

    def mlp_set(self, params, out_mean=None, out_std=None) -> int:
        n = params.numel() if hasattr(params, "numel") else params.size
        return _check(self.lib.klecgc_mlp_set(self.h, _ptr(params, np.float32), n,
                                              _ptr(out_mean, np.float32),
                                              _ptr(out_std, np.float32)))

    def mlp_get(self, params=None, out_mean=None, out_std=None) -> int:
        return _check(self.lib.klecgc_mlp_get(self.h, _ptr(params, np.float32),
                                              _ptr(out_mean, np.float32),
                                              _ptr(out_std, np.float32), None))

    def mlp_loss_grad(self, xi, targets, B, grad_out=None, stream=None) -> float:
        loss = ctypes.c_double()
        _check(self.lib.klecgc_mlp_loss_grad(self.h, _ptr(xi, np.float64),
                                             _ptr(targets, np.float32), B, ctypes.byref(loss),
                                             _ptr(grad_out, np.float32), _stream(stream)))
        return loss.value

    def mlp_train(self, xi, targets, n, epochs, batch, lr, lr_final, seed, fit_norm=True,
                  stream=None) -> np.ndarray:
        losses = np.zeros(epochs, dtype=np.float32)
        _check(self.lib.klecgc_mlp_train(self.h, _ptr(xi, np.float64), _ptr(targets, np.float32),
                                         n, epochs, batch, lr, lr_final, seed,
                                         1 if fit_norm else 0, losses.ctypes.data,
                                         _stream(stream)))
        return losses

    def mlp_guess(self, xi, S, U0_out, stream=None) -> int:
        return _check(self.lib.klecgc_mlp_guess(self.h, _ptr(xi, np.float64), S,
                                                _ptr(U0_out, np.float64), _stream(stream)),
                      (OK, E_NONFINITE))

    def downsample(self, U, S, N, T_out, stream=None) -> int:
        return _check(self.lib.klecgc_downsample(self.h, _ptr(U, np.float64), S, N,
                                                 _ptr(T_out, np.float32), _stream(stream)))

    def mlp_set_residual(self, residual) -> int:
        """1: the network corrects the gPC surrogate guess; 0: it is the guess."""
        return _check(self.lib.klecgc_mlp_set_residual(self.h, int(residual)))

    def mlp_targets(self, xi, U, S, T_out, stream=None) -> int:
        """Training targets of the current mode at the 64 network points."""
        return _check(self.lib.klecgc_mlp_targets(self.h, _ptr(xi, np.float64),
                                                  _ptr(U, np.float64), S,
                                                  _ptr(T_out, np.float32), _stream(stream)))

    def reference_noalloc(self, xi, S, N, J, U_out, stream=None) -> int:
        """klecgc_reference without device allocation (device arrays only)."""
        return _check(self.lib.klecgc_reference_noalloc(self.h, _ptr(xi, np.float64), S, N, J,
                                                         _ptr(U_out, np.float64),
                                                         _stream(stream)))
