"""Python binding of the C ABI in include/asdsm.h (argument marshalling only).

Every step of ASDSM runs in libasdsm.so on the GPU; this module only passes
device pointers of PyTorch tensors, the current CUDA stream and plain
structs.  It raises if the library is missing: there is no CPU fallback.

    import torch
    from paper_2303_01163_gb300 import asdsm
    solver = asdsm.Solver(N=1025, mc=64, alpha=(1, 1), beta=(1, 1))
    u = torch.zeros(N, N, dtype=torch.float64, device="cuda")   # ring = g
    stats = solver.solve(s, u)                                  # s: (N, N) float64 on the GPU
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libasdsm.so")

OK = 0
ERR_INVALID = -1
ERR_CUDA = -2
ERR_OOM = -3
ERR_NAN = -4
NOT_CONVERGED = -5
STAGNATED = -6
ERR_RANGE = -7

FP64 = 0
MIXED = 1

MESH_FC, MESH_CF, MESH_CC, MESH_HOLES, MESH_HOLES_HOMOGENEOUS = 0, 1, 2, 3, 4
# 3D (asdsm_submesh_solve with d = 3): plane families, line families, coarse mesh, cube holes.
MESH3_PLANE, MESH3_LINE, MESH3_COARSE, MESH3_HOLES, MESH3_FILL = 0, 3, 6, 7, 8


class Desc(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("n", ctypes.c_int32), ("mc", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("alpha", ctypes.c_double * 3), ("beta", ctypes.c_double * 3)]


class Opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_sweeps", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("accel_m", ctypes.c_int32), ("skip_initial_guess", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("hole_fix_ratio", ctypes.c_double), ("hole_fix_growth", ctypes.c_double),
                ("stagnation_window", ctypes.c_int32), ("sweep_graph", ctypes.c_int32),
                ("stagnation_factor", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int32), ("status", ctypes.c_int32), ("hole_fixes", ctypes.c_int32),
                ("fixed_shift", ctypes.c_int32), ("rel_res", ctypes.c_double), ("rel_res0", ctypes.c_double),
                ("setup_ms", ctypes.c_double), ("solve_ms", ctypes.c_double), ("launches", ctypes.c_int64),
                ("rel_res_fp64", ctypes.c_double), ("hole_res_max", ctypes.c_double),
                ("rescales", ctypes.c_int32), ("pad_", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class KProf(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_int64), ("calls", ctypes.c_int64),
                ("ms", ctypes.c_double), ("bytes", ctypes.c_double), ("flops", ctypes.c_double)]


_lib = None


def library_path() -> str:
    return _LIB_PATH


def load() -> ctypes.CDLL:
    """Load libasdsm.so (built by __graft_entry__.build()); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"libasdsm.so not built ({_LIB_PATH}); run __graft_entry__.build() first")
    lib = ctypes.CDLL(_LIB_PATH)
    P = ctypes.c_void_p
    lib.asdsm_default_opts.argtypes = [ctypes.POINTER(Opts)]
    lib.asdsm_default_opts.restype = None
    lib.asdsm_setup.argtypes = [ctypes.POINTER(Desc), ctypes.POINTER(Opts), P, ctypes.POINTER(P)]
    lib.asdsm_setup.restype = ctypes.c_int
    lib.asdsm_set_opts.argtypes = [P, ctypes.POINTER(Opts)]
    lib.asdsm_set_opts.restype = ctypes.c_int
    lib.asdsm_autotune.argtypes = [P, ctypes.c_int]
    lib.asdsm_autotune.restype = ctypes.c_int
    lib.asdsm_tune_get.argtypes = [P, ctypes.POINTER(ctypes.c_int32), ctypes.c_int]
    lib.asdsm_tune_get.restype = ctypes.c_int
    lib.asdsm_tune_set.argtypes = [P, ctypes.POINTER(ctypes.c_int32), ctypes.c_int]
    lib.asdsm_tune_set.restype = ctypes.c_int
    lib.asdsm_real_schur.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double)]
    lib.asdsm_real_schur.restype = ctypes.c_int
    lib.asdsm_bcr_tail_map.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_double)]
    lib.asdsm_bcr_tail_map.restype = ctypes.c_int
    lib.asdsm_selftest_wait_timeout.argtypes = [P, ctypes.c_longlong]
    lib.asdsm_selftest_wait_timeout.restype = ctypes.c_int
    lib.asdsm_tune_check.argtypes = [ctypes.POINTER(ctypes.c_int32), ctypes.c_int]
    lib.asdsm_tune_check.restype = ctypes.c_int
    lib.asdsm_solve.argtypes = [P, P, P, ctypes.POINTER(Stats)]
    lib.asdsm_solve.restype = ctypes.c_int
    lib.asdsm_initial_guess.argtypes = [P, P, P]
    lib.asdsm_initial_guess.restype = ctypes.c_int
    lib.asdsm_residual.argtypes = [P, P, P, P, ctypes.POINTER(ctypes.c_double)]
    lib.asdsm_residual.restype = ctypes.c_int
    lib.asdsm_submesh_solve.argtypes = [P, ctypes.c_int, P, P]
    lib.asdsm_submesh_solve.restype = ctypes.c_int
    lib.asdsm_history.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.c_int]
    lib.asdsm_history.restype = ctypes.c_int
    lib.asdsm_hole_extension_operator.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                                  ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    lib.asdsm_hole_extension_operator.restype = ctypes.c_int
    lib.asdsm_hole_extension_operator_3d.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    lib.asdsm_hole_extension_operator_3d.restype = ctypes.c_int
    lib.asdsm_profile.argtypes = [P, ctypes.c_int]
    lib.asdsm_profile.restype = ctypes.c_int
    lib.asdsm_profile_read.argtypes = [P, ctypes.POINTER(KProf), ctypes.c_int]
    lib.asdsm_profile_read.restype = ctypes.c_int
    lib.asdsm_launch_count.argtypes = []
    lib.asdsm_launch_count.restype = ctypes.c_int64
    lib.asdsm_residual_noalloc.argtypes = [ctypes.POINTER(Desc), P, P, P, ctypes.POINTER(ctypes.c_double), P]
    lib.asdsm_residual_noalloc.restype = ctypes.c_int
    lib.asdsm_noalloc_last_error.argtypes = []
    lib.asdsm_noalloc_last_error.restype = ctypes.c_char_p
    lib.asdsm_destroy.argtypes = [P]
    lib.asdsm_destroy.restype = None
    lib.asdsm_setup_batch.argtypes = [ctypes.POINTER(Desc), ctypes.c_int, ctypes.POINTER(Opts), P, ctypes.POINTER(P)]
    lib.asdsm_setup_batch.restype = ctypes.c_int
    lib.asdsm_batch_count.argtypes = [P]
    lib.asdsm_batch_count.restype = ctypes.c_int
    lib.asdsm_set_opts_batch.argtypes = [P, ctypes.POINTER(Opts)]
    lib.asdsm_set_opts_batch.restype = ctypes.c_int
    lib.asdsm_autotune_batch.argtypes = [P, ctypes.c_int]
    lib.asdsm_autotune_batch.restype = ctypes.c_int
    lib.asdsm_solve_batch.argtypes = [P, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(Stats)]
    lib.asdsm_solve_batch.restype = ctypes.c_int
    lib.asdsm_batch_history.argtypes = [P, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int]
    lib.asdsm_batch_history.restype = ctypes.c_int
    lib.asdsm_destroy_batch.argtypes = [P]
    lib.asdsm_destroy_batch.restype = None
    lib.asdsm_cnn_param_count.argtypes = []
    lib.asdsm_cnn_param_count.restype = ctypes.c_int
    lib.asdsm_cnn_create.argtypes = [ctypes.POINTER(ctypes.c_float), ctypes.c_int, ctypes.c_int, ctypes.POINTER(P)]
    lib.asdsm_cnn_create.restype = ctypes.c_int
    lib.asdsm_cnn_get_params.argtypes = [P, ctypes.POINTER(ctypes.c_float), ctypes.c_int]
    lib.asdsm_cnn_get_params.restype = ctypes.c_int
    lib.asdsm_cnn_set_params.argtypes = [P, ctypes.POINTER(ctypes.c_float), ctypes.c_int]
    lib.asdsm_cnn_set_params.restype = ctypes.c_int
    lib.asdsm_cnn_forward.argtypes = [P, P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P]
    lib.asdsm_cnn_forward.restype = ctypes.c_int
    lib.asdsm_cnn_backward.argtypes = [P, P, P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float), P]
    lib.asdsm_cnn_backward.restype = ctypes.c_int
    lib.asdsm_cnn_adam.argtypes = [P, ctypes.c_float, P]
    lib.asdsm_cnn_adam.restype = ctypes.c_int
    lib.asdsm_cnn_last_error.argtypes = []
    lib.asdsm_cnn_last_error.restype = ctypes.c_char_p
    lib.asdsm_cnn_destroy.argtypes = [P]
    lib.asdsm_cnn_destroy.restype = None
    lib.asdsm_attach_cnn.argtypes = [P, P]
    lib.asdsm_attach_cnn.restype = ctypes.c_int
    lib.asdsm_cnn_directions.argtypes = [P]
    lib.asdsm_cnn_directions.restype = ctypes.c_int
    lib.asdsm_correction.argtypes = [P, P, P, P, P, ctypes.c_int]
    lib.asdsm_correction.restype = ctypes.c_int
    lib.asdsm_strerror.argtypes = [ctypes.c_int]
    lib.asdsm_strerror.restype = ctypes.c_char_p
    lib.asdsm_last_error.argtypes = []
    lib.asdsm_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


class AsdsmError(RuntimeError):
    def __init__(self, code: int, what: str):
        lib = load()
        msg = lib.asdsm_strerror(code).decode()
        extra = lib.asdsm_last_error().decode()
        super().__init__(f"{what}: {msg} ({code})" + (f": {extra}" if extra else ""))
        self.code = code


def default_opts() -> Opts:
    o = Opts()
    load().asdsm_default_opts(ctypes.byref(o))
    return o


def _ptr(t, dtype_name="float64"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if str(t.dtype) != f"torch.{dtype_name}":
        raise TypeError(f"expected torch.{dtype_name}, got {t.dtype}")
    if not t.is_contiguous():
        raise TypeError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def residual_noalloc(N: int, alpha, beta, s, u, r=None, stream=None) -> float:
    """asdsm_residual_noalloc: residual and ||r||/||b|| with no device allocation
    (2D: two alpha/beta per axis and N*N grids; 3D: three and N*N*N grids)."""
    import torch
    lib = load()
    d = Desc()
    dim = len(alpha)
    d.d, d.n = dim, int(N)
    for q in range(dim):
        d.alpha[q] = float(alpha[q])
        d.beta[q] = float(beta[q])
    if stream is None:
        stream = torch.cuda.current_stream()
    rel = ctypes.c_double()
    rc = lib.asdsm_residual_noalloc(ctypes.byref(d), _ptr(s), _ptr(u), _ptr(r) if r is not None else None,
                                    ctypes.byref(rel), ctypes.c_void_p(stream.cuda_stream))
    if rc != OK:
        raise RuntimeError(f"asdsm_residual_noalloc: {lib.asdsm_strerror(rc).decode()} ({rc}): "
                           f"{lib.asdsm_noalloc_last_error().decode()}")
    return rel.value


def hole_extension_operator_3d(N: int, mc: int, alpha, beta):
    """G of asdsm_hole_extension_operator_3d as a (C^3, 6 C^2) numpy array (host, no GPU)."""
    import numpy as np
    lib = load()
    C = (N - 1) // mc - 1
    G = np.zeros((C ** 3, 6 * C * C), dtype=np.float64)
    a = (ctypes.c_double * 3)(*[float(x) for x in alpha])
    b = (ctypes.c_double * 3)(*[float(x) for x in beta])
    rc = lib.asdsm_hole_extension_operator_3d(int(N), int(mc), a, b, G.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != OK:
        raise AsdsmError(rc, "asdsm_hole_extension_operator_3d")
    return G


def hole_extension_operator(N: int, mc: int, alpha, beta):
    """G of asdsm_hole_extension_operator as a (C*C, 4C) numpy array (host, no GPU)."""
    import numpy as np
    lib = load()
    C = (N - 1) // mc - 1
    G = np.zeros((C * C, 4 * C), dtype=np.float64)
    a = (ctypes.c_double * 2)(*[float(x) for x in alpha])
    b = (ctypes.c_double * 2)(*[float(x) for x in beta])
    rc = lib.asdsm_hole_extension_operator(int(N), int(mc), a, b, G.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != OK:
        raise AsdsmError(rc, "asdsm_hole_extension_operator")
    return G


@dataclass
class SolveResult:
    status: int
    stats: dict
    history: list


class Solver:
    """One problem of eq. (1.1) on an N x N grid (the handle of asdsm_setup),
    or, with three alpha and beta values, on an N x N x N grid (the 3D
    extension, Section 3.5)."""

    def __init__(self, N: int, mc: int, alpha, beta, *, precision: int = MIXED, tol: float = 1e-10,
                 max_sweeps: int = 500, accel_m: int = 8, seed: int = 0, stream=None, **opt_overrides):
        import torch
        lib = load()
        self._lib = lib
        self.N, self.mc = int(N), int(mc)
        d = Desc()
        self.dim = len(alpha)
        if self.dim not in (2, 3) or len(beta) != self.dim:
            raise ValueError("alpha and beta need 2 (2D) or 3 (3D) values each")
        d.d = self.dim
        d.n = self.N
        d.mc = self.mc
        for q in range(self.dim):
            d.alpha[q] = float(alpha[q])
            d.beta[q] = float(beta[q])
        o = default_opts()
        o.tol, o.max_sweeps, o.precision, o.accel_m, o.seed = tol, max_sweeps, precision, accel_m, seed
        for k, v in opt_overrides.items():
            setattr(o, k, v)
        self.opts = o
        if stream is None:
            stream = torch.cuda.current_stream()
        self._stream = stream
        h = ctypes.c_void_p()
        rc = lib.asdsm_setup(ctypes.byref(d), ctypes.byref(o), ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h))
        if rc != OK:
            raise AsdsmError(rc, "asdsm_setup")
        self._h = h

    def set_opts(self, **kw):
        for k, v in kw.items():
            setattr(self.opts, k, v)
        rc = self._lib.asdsm_set_opts(self._h, ctypes.byref(self.opts))
        if rc != OK:
            raise AsdsmError(rc, "asdsm_set_opts")

    def autotune(self, precision=None):
        """Time and keep the fastest launch shapes for this handle (asdsm_autotune)."""
        prec = self.opts.precision if precision is None else precision
        rc = self._lib.asdsm_autotune(self._h, prec)
        if rc != OK:
            raise AsdsmError(rc, "asdsm_autotune")

    def attach_cnn(self, net):
        """Use a Cnn as the learned correction (None detaches); keep `net` alive meanwhile."""
        self._cnn = net
        rc = self._lib.asdsm_attach_cnn(self._h, net._h if net is not None else None)
        if rc != OK:
            raise AsdsmError(rc, "asdsm_attach_cnn")

    def cnn_directions(self) -> int:
        return self._lib.asdsm_cnn_directions(self._h)

    def correction(self, s, u, k: int = 0):
        """(r, e) of iterate u as FP32 N x N tensors (asdsm_correction)."""
        import torch
        r = torch.empty((self.N, self.N), dtype=torch.float32, device=u.device)
        e = torch.empty_like(r)
        rc = self._lib.asdsm_correction(self._h, _ptr(s), _ptr(u), _ptr(r, "float32"), _ptr(e, "float32"), int(k))
        if rc != OK:
            raise AsdsmError(rc, "asdsm_correction")
        return r, e

    def tune_state(self) -> list:
        buf = (ctypes.c_int32 * 256)()
        n = self._lib.asdsm_tune_get(self._h, buf, 256)
        if n < 0:
            raise AsdsmError(n, "asdsm_tune_get")
        return [int(buf[i]) for i in range(n)]

    def set_tune_state(self, values):
        arr = (ctypes.c_int32 * len(values))(*values)
        rc = self._lib.asdsm_tune_set(self._h, arr, len(values))
        if rc != OK:
            raise AsdsmError(rc, "asdsm_tune_set")

    def solve(self, s, u, check: bool = True) -> SolveResult:
        st = Stats()
        rc = self._lib.asdsm_solve(self._h, _ptr(s), _ptr(u), ctypes.byref(st))
        if rc not in (OK, NOT_CONVERGED, STAGNATED) and check:
            raise AsdsmError(rc, "asdsm_solve")
        return SolveResult(rc, st.as_dict(), self.history())

    def initial_guess(self, s, u):
        rc = self._lib.asdsm_initial_guess(self._h, _ptr(s), _ptr(u))
        if rc != OK:
            raise AsdsmError(rc, "asdsm_initial_guess")

    def residual(self, s, u, r=None) -> float:
        rel = ctypes.c_double()
        rc = self._lib.asdsm_residual(self._h, _ptr(s), _ptr(u), _ptr(r) if r is not None else None, ctypes.byref(rel))
        if rc != OK:
            raise AsdsmError(rc, "asdsm_residual")
        return rel.value

    def submesh_solve(self, mesh: int, inp, out):
        rc = self._lib.asdsm_submesh_solve(self._h, int(mesh), _ptr(inp), _ptr(out))
        if rc != OK:
            raise AsdsmError(rc, "asdsm_submesh_solve")

    def profile(self, enable: bool = True):
        rc = self._lib.asdsm_profile(self._h, 1 if enable else 0)
        if rc != OK:
            raise AsdsmError(rc, "asdsm_profile")

    def profile_read(self) -> dict:
        buf = (KProf * 16)()
        n = self._lib.asdsm_profile_read(self._h, buf, 16)
        if n < 0:
            raise AsdsmError(n, "asdsm_profile_read")
        return {buf[i].name.decode(): {"launches": buf[i].launches, "calls": buf[i].calls, "ms": buf[i].ms,
                                       "bytes": buf[i].bytes, "flops": buf[i].flops} for i in range(n)}

    def history(self) -> list:
        cap = 100000
        buf = (ctypes.c_double * cap)()
        n = self._lib.asdsm_history(self._h, buf, cap)
        if n < 0:
            raise AsdsmError(n, "asdsm_history")
        return [buf[i] for i in range(n)]

    def close(self):
        if getattr(self, "_h", None):
            self._lib.asdsm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class BatchSolver:
    """Many independent problems of eq. (1.1) (asdsm_setup_batch): problems is a
    list of (N, mc, alpha, beta); solve takes lists of device tensors."""

    def __init__(self, problems, *, precision: int = MIXED, tol: float = 1e-10, max_sweeps: int = 500,
                 accel_m: int = 8, seed: int = 0, stream=None, **opt_overrides):
        import torch
        lib = load()
        self._lib = lib
        n = len(problems)
        descs = (Desc * n)()
        self.sizes = []
        for i, (N, mc, alpha, beta) in enumerate(problems):
            descs[i].d, descs[i].n, descs[i].mc = 2, int(N), int(mc)
            for q in range(2):
                descs[i].alpha[q] = float(alpha[q])
                descs[i].beta[q] = float(beta[q])
            self.sizes.append(int(N))
        o = default_opts()
        o.tol, o.max_sweeps, o.precision, o.accel_m, o.seed = tol, max_sweeps, precision, accel_m, seed
        for k, v in opt_overrides.items():
            setattr(o, k, v)
        self.opts = o
        if stream is None:
            stream = torch.cuda.current_stream()
        self._stream = stream
        h = ctypes.c_void_p()
        rc = lib.asdsm_setup_batch(descs, n, ctypes.byref(o), ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h))
        if rc != OK:
            raise AsdsmError(rc, "asdsm_setup_batch")
        self._h = h
        self.count = lib.asdsm_batch_count(h)

    def set_opts(self, **kw):
        for k, v in kw.items():
            setattr(self.opts, k, v)
        rc = self._lib.asdsm_set_opts_batch(self._h, ctypes.byref(self.opts))
        if rc != OK:
            raise AsdsmError(rc, "asdsm_set_opts_batch")

    def autotune(self, precision=None):
        prec = self.opts.precision if precision is None else precision
        rc = self._lib.asdsm_autotune_batch(self._h, prec)
        if rc != OK:
            raise AsdsmError(rc, "asdsm_autotune_batch")

    def solve(self, s_list, u_list, check: bool = True):
        """Returns (status, [stats dict per instance])."""
        n = self.count
        if len(s_list) != n or len(u_list) != n:
            raise ValueError("one s and one u per instance")
        for i in range(n):
            N = self.sizes[i]
            if s_list[i].numel() != N * N or u_list[i].numel() != N * N:
                raise ValueError(f"instance {i}: expected {N}x{N} grids")
        VP = ctypes.c_void_p
        sp = (VP * n)(*[_ptr(t) for t in s_list])
        up = (VP * n)(*[_ptr(t) for t in u_list])
        st = (Stats * n)()
        rc = self._lib.asdsm_solve_batch(self._h, sp, up, st)
        if check and rc not in (OK, NOT_CONVERGED, STAGNATED):
            raise AsdsmError(rc, "asdsm_solve_batch")
        return rc, [st[i].as_dict() for i in range(n)]

    def history(self, index: int) -> list:
        cap = 100000
        buf = (ctypes.c_double * cap)()
        k = self._lib.asdsm_batch_history(self._h, int(index), buf, cap)
        if k < 0:
            raise AsdsmError(k, "asdsm_batch_history")
        return [buf[i] for i in range(k)]

    def close(self):
        if getattr(self, "_h", None):
            self._lib.asdsm_destroy_batch(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Cnn:
    """The learned-correction network (asdsm_cnn_*): device FP32 NCHW tensors in and out."""

    def __init__(self, params, bf16: bool = True, stream=None):
        import numpy as np
        import torch
        lib = load()
        self._lib = lib
        self.n = lib.asdsm_cnn_param_count()
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != self.n:
            raise ValueError(f"expected {self.n} parameters")
        h = ctypes.c_void_p()
        rc = lib.asdsm_cnn_create(p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), self.n, 1 if bf16 else 0,
                                  ctypes.byref(h))
        if rc != OK:
            raise AsdsmError(rc, "asdsm_cnn_create")
        self._h = h
        self._stream = stream if stream is not None else torch.cuda.current_stream()

    def params(self):
        import numpy as np
        out = np.empty(self.n, dtype=np.float32)
        rc = self._lib.asdsm_cnn_get_params(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), self.n)
        if rc != OK:
            raise AsdsmError(rc, "asdsm_cnn_get_params")
        return out

    def set_params(self, params):
        import numpy as np
        p = np.ascontiguousarray(params, dtype=np.float32)
        rc = self._lib.asdsm_cnn_set_params(self._h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), self.n)
        if rc != OK:
            raise AsdsmError(rc, "asdsm_cnn_set_params")

    def forward(self, x):
        import torch
        B, C, H, W = x.shape
        y = torch.empty((B, 1, H, W), dtype=torch.float32, device=x.device)
        rc = self._lib.asdsm_cnn_forward(self._h, _ptr(x, "float32"), _ptr(y, "float32"), B, H, W,
                                         ctypes.c_void_p(self._stream.cuda_stream))
        if rc != OK:
            raise AsdsmError(rc, "asdsm_cnn_forward")
        return y

    def backward(self, x, t, want_grad: bool = False, weights=None):
        """Returns (loss, gradient as numpy or None); weights: optional (B,1,H,W) per-pixel loss weights."""
        import numpy as np
        B, C, H, W = x.shape
        loss = ctypes.c_double()
        g = np.empty(self.n, dtype=np.float32) if want_grad else None
        wp = _ptr(weights, "float32") if weights is not None else None
        rc = self._lib.asdsm_cnn_backward(self._h, _ptr(x, "float32"), _ptr(t, "float32"), wp, B, H, W, ctypes.byref(loss),
                                          g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)) if want_grad else None,
                                          ctypes.c_void_p(self._stream.cuda_stream))
        if rc != OK:
            raise AsdsmError(rc, "asdsm_cnn_backward")
        return loss.value, g

    def adam(self, lr: float):
        rc = self._lib.asdsm_cnn_adam(self._h, float(lr), ctypes.c_void_p(self._stream.cuda_stream))
        if rc != OK:
            raise AsdsmError(rc, "asdsm_cnn_adam")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.asdsm_cnn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
