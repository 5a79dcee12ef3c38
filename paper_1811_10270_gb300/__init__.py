"""Python binding of the shbim C ABI (include/shbim.h): argument marshalling only.

Every computation runs in the CUDA library libshbim.so built in-tree by build.py. There is no
CPU fallback: if the library is missing or cannot be loaded, every call raises.
Tensors passed in must be CUDA float64 tensors, contiguous, on the current device; the
current torch stream is passed to the library.
"""
from __future__ import annotations

import ctypes
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libshbim.so")

FP64 = 0
FP32_COMP = 1
DF64 = 2
LAPLACE_DL = 0
LAPLACE_SL = 1
OUT_GRID = 0
OUT_COEF = 1
SHT_INVERSE = 0
SHT_FORWARD = 1
GRID_BASE = 0
GRID_UP = 1
SYS_ELECTRIC = 0
SYS_STOKES = 1
SYS_DIFFUSION = 2
TC_FOURIER = 1
TC_ROTATION = 2
TC_LEGENDRE = 4
TC_ALL = 7
CONTINUE = 0
CONVERGED = 1
EOS_LANGMUIR = 0
EOS_LINEAR = 1

EXPORTS = [
    "shbim_create", "shbim_destroy", "shbim_last_error", "shbim_set_precision", "shbim_set_R",
    "shbim_set_drops", "shbim_sizes", "shbim_target_geometry", "shbim_sht", "shbim_eval_electric",
    "shbim_eval_stokes", "shbim_gmres_begin", "shbim_gmres_step", "shbim_gmres_finish",
    "shbim_gmres_solve", "shbim_launch_count", "shbim_electric_rhs", "shbim_set_timing",
    "shbim_kernel_stats", "shbim_gmres_solve_refined", "shbim_pairs_laplace_noalloc",
    "shbim_rates", "shbim_step", "shbim_operator_applications", "shbim_set_near", "shbim_near_pairs",
    "shbim_mlp_create", "shbim_mlp_destroy", "shbim_mlp_set_layer", "shbim_mlp_get_layer",
    "shbim_mlp_forward", "shbim_mlp_train_step", "shbim_electric_warm_start", "shbim_mlp_set_input_affine",
    "shbim_set_graphs", "shbim_set_concurrency", "shbim_pair_queue", "shbim_set_pair_queue", "shbim_laplace_beltrami", "shbim_set_diffusion",
    "shbim_set_autotune", "shbim_pair_shape", "shbim_set_pair_shape", "shbim_probe_peak",
    "shbim_set_outer_precision", "shbim_set_rows_precision", "shbim_set_tensor_cores",
    "shbim_near_min_distance", "shbim_set_wait_limit", "shbim_check_wait", "shbim_set_self_precision", "shbim_set_oneshot_precision",
    "shbim_kernel_work", "shbim_warm_start_feature_count", "shbim_warm_start_features", "shbim_learned_guess",
    "shbim_set_warm_start", "shbim_stokes_rhs", "shbim_set_device_gmres", "shbim_reparametrize",
    "shbim_set_field_shape", "shbim_set_equation_of_state", "shbim_set_quantized_pairs",
    "shbim_set_stokes_preconditioner",
]
PROBE_FFMA = 0
PROBE_DFMA = 1
PROBE_RSQRT = 2
PROBE_HMMA_BF16 = 3
PROBE_DMMA_F64 = 4
NOALLOC_MAX_TARGETS = 1 << 21
ERR_ARG = -1
ERR_CUDA = -2
ERR_TIMEOUT = -5
K_SELF_WEIGHTS = 0
K_SELF_ANALYSIS = 1
K_PAIRS = 2
K_SELF_GEMV = 3
K_SHT = 4
K_SELF_ROTATION = 5
K_PAIRS_FP64CLASS = 6
K_NEAR = 7
K_COUNT = 8


class ShbimError(RuntimeError):
    pass


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("gmres_restart", ctypes.c_int),
                ("gmres_tol", ctypes.c_double), ("gmres_maxiter", ctypes.c_int),
                ("R", ctypes.c_double)]


class Phys(ctypes.Structure):
    """shbim_phys: R, Q, Ca_E, Langmuir beta and x_s, far field E_u + E_q (x, -y, 0), the
    inner tolerance of the mixed-precision solves and the surfactant Peclet number (0 or
    infinity: no diffusion)."""
    _fields_ = [("R", ctypes.c_double), ("Q", ctypes.c_double), ("Ca_E", ctypes.c_double),
                ("beta", ctypes.c_double), ("x_s", ctypes.c_double), ("E_u", ctypes.c_double * 3),
                ("E_q", ctypes.c_double), ("inner_tol", ctypes.c_double), ("Pe", ctypes.c_double)]


def phys(R=2.0, Q=0.5, Ca_E=0.1, beta=0.2, x_s=0.5, E_u=(0.0, 0.0, 1.0), E_q=0.0, inner_tol=1e-5,
         Pe=math.inf):
    return Phys(R, Q, Ca_E, beta, x_s, (ctypes.c_double * 3)(*E_u), E_q, inner_tol, Pe)


_lib = None


def lib():
    """Load libshbim.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ShbimError("libshbim.so is not built (run paper_1811_10270_gb300.build.build())")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    P = ctypes.POINTER
    sig = {
        "shbim_create": (i32, [P(Opts), P(vp)]),
        "shbim_destroy": (i32, [vp]),
        "shbim_last_error": (ctypes.c_char_p, [vp]),
        "shbim_set_precision": (i32, [vp, i32]),
        "shbim_set_R": (i32, [vp, dp]),
        "shbim_set_drops": (i32, [vp, i32, P(ctypes.c_int32), P(dp), vp, vp]),
        "shbim_sizes": (i32, [vp, P(i64), P(i64), P(i64)]),
        "shbim_target_geometry": (i32, [vp, vp, vp]),
        "shbim_sht": (i32, [vp, i32, i32, i32, P(ctypes.c_int32), vp, vp, vp]),
        "shbim_eval_electric": (i32, [vp, i32, vp, vp, i32, vp]),
        "shbim_eval_stokes": (i32, [vp, vp, vp, vp, i32, vp]),
        "shbim_gmres_begin": (i32, [vp, i32, vp, vp, vp]),
        "shbim_gmres_step": (i32, [vp, P(dp), vp]),
        "shbim_gmres_finish": (i32, [vp, vp, P(i32), vp]),
        "shbim_gmres_solve": (i32, [vp, i32, vp, vp, vp, P(i32), P(dp), vp]),
        "shbim_launch_count": (i64, [vp]),
        "shbim_electric_rhs": (i32, [vp, P(dp), dp, vp, vp]),
        "shbim_set_timing": (i32, [vp, i32]),
        "shbim_kernel_stats": (i32, [vp, i32, P(dp), P(i64)]),
        "shbim_gmres_solve_refined": (i32, [vp, i32, vp, vp, vp, dp, i32, P(i32), P(i32), P(dp), vp]),
        "shbim_pairs_laplace_noalloc": (i32, [i32, vp, i64, vp, i64, vp, vp]),
        "shbim_rates": (i32, [vp, P(Phys), vp, vp, vp, P(i32), vp]),
        "shbim_step": (i32, [vp, P(Phys), vp, vp, dp, vp, vp, P(dp), P(i32), vp]),
        "shbim_operator_applications": (i64, [vp]),
        "shbim_set_near": (i32, [vp, i32]),
        "shbim_set_graphs": (i32, [vp, i32]),
        "shbim_set_concurrency": (i32, [vp, i32]),
        "shbim_pair_queue": (i32, [vp, i32]),
        "shbim_set_pair_queue": (i32, [vp, i32, i32]),
        "shbim_set_autotune": (i32, [vp, i32]),
        "shbim_set_outer_precision": (i32, [vp, i32]),
        "shbim_set_rows_precision": (i32, [vp, i32]),
        "shbim_set_tensor_cores": (i32, [vp, i32]),
        "shbim_pair_shape": (i32, [vp, i32, P(i32), P(i32)]),
        "shbim_probe_peak": (i32, [i32, i64, P(dp), P(dp), vp]),
        "shbim_set_pair_shape": (i32, [vp, i32, i32, i32]),
        "shbim_laplace_beltrami": (i32, [vp, vp, vp, vp]),
        "shbim_set_diffusion": (i32, [vp, dp]),
        "shbim_mlp_create": (i32, [i32, P(ctypes.c_int32), i32, P(vp)]),
        "shbim_mlp_destroy": (i32, [vp]),
        "shbim_mlp_set_layer": (i32, [vp, i32, vp, vp]),
        "shbim_mlp_get_layer": (i32, [vp, i32, vp, vp, vp, vp]),
        "shbim_mlp_set_input_affine": (i32, [vp, vp, vp]),
        "shbim_mlp_forward": (i32, [vp, i32, vp, vp, vp]),
        "shbim_mlp_train_step": (i32, [vp, i32, vp, vp, ctypes.c_float, i32, P(dp), vp]),
        "shbim_electric_warm_start": (i32, [vp, vp, vp, vp, vp, vp]),
        "shbim_near_pairs": (i32, [vp]),
        "shbim_near_min_distance": (i32, [vp, P(dp), P(dp)]),
        "shbim_set_wait_limit": (i32, [vp, dp]),
        "shbim_check_wait": (i32, [vp, i32, vp]),
        "shbim_set_self_precision": (i32, [vp, i32]),
        "shbim_set_oneshot_precision": (i32, [vp, i32]),
        "shbim_kernel_work": (i32, [vp, i32, P(dp)]),
        "shbim_warm_start_feature_count": (i64, [vp]),
        "shbim_warm_start_features": (i32, [vp, vp, vp, P(Phys), vp, vp]),
        "shbim_learned_guess": (i32, [vp, vp, vp, vp, vp, vp, vp]),
        "shbim_set_warm_start": (i32, [vp, vp]),
        "shbim_stokes_rhs": (i32, [vp, P(Phys), vp, vp, vp, vp]),
        "shbim_set_device_gmres": (i32, [vp, i32]),
        "shbim_reparametrize": (i32, [vp, i32, dp, dp, vp, vp, P(dp), vp]),
        "shbim_set_field_shape": (i32, [vp, P(dp)]),
        "shbim_set_equation_of_state": (i32, [vp, i32]),
        "shbim_set_quantized_pairs": (i32, [vp, i32]),
        "shbim_set_stokes_preconditioner": (i32, [vp, i32]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _ptr(t):
    if t is None:
        return None
    import torch
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ShbimError("expected a contiguous CUDA float64 tensor")
    return ctypes.c_void_p(t.data_ptr())


def _ptr32(t):
    import torch
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise ShbimError("expected a contiguous CUDA float32 tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def pairs_laplace_noalloc(which: int, tgt, src, out) -> int:
    """shbim_pairs_laplace_noalloc: FP64 Laplace pair sum of src (4 x n_src: x, y, z, strength)
    at tgt (6 x n_tgt: x, y, z, nx, ny, nz) into out (n_tgt), without any device allocation.
    The counts come from out and src; the tensors must hold them (the C ABI cannot check).
    Returns the library's status code (0 on success)."""
    L = lib()
    nt = out.numel()
    ns = src.numel() // 4
    if tgt.numel() < 6 * nt or src.numel() != 4 * ns:
        raise ShbimError("pairs_laplace_noalloc: tgt must hold 6 x n_tgt and src 4 x n_src doubles")
    return int(L.shbim_pairs_laplace_noalloc(int(which), _ptr(tgt), nt, _ptr(src), ns, _ptr(out),
                                             _stream()))


class Context:
    """One shbim context (shbim_create / shbim_destroy)."""

    def __init__(self, precision: int = FP64, gmres_restart: int = 50, gmres_tol: float = 1e-8,
                 gmres_maxiter: int = 1000, R: float = 1.0):
        L = lib()
        self._L = L
        o = Opts(precision, gmres_restart, gmres_tol, gmres_maxiter, R)
        h = ctypes.c_void_p()
        rc = L.shbim_create(ctypes.byref(o), ctypes.byref(h))
        if rc != 0:
            raise ShbimError("shbim_create failed (%d)" % rc)
        self._h = h
        self.p = []

    def close(self):
        if getattr(self, "_h", None):
            self._L.shbim_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc < 0:
            msg = self._L.shbim_last_error(self._h).decode()
            raise ShbimError("%s failed (%d): %s" % (what, rc, msg))
        return rc

    # ---------------------------------------------------------------- set-up
    def set_precision(self, precision: int):
        self._check(self._L.shbim_set_precision(self._h, precision), "shbim_set_precision")

    def set_R(self, R: float):
        self._check(self._L.shbim_set_R(self._h, float(R)), "shbim_set_R")

    def set_drops(self, p_list, xcoef, lam_list=None):
        n = len(p_list)
        P = (ctypes.c_int32 * n)(*[int(p) for p in p_list])
        lam = None if lam_list is None else (ctypes.c_double * n)(*[float(x) for x in lam_list])
        self._check(self._L.shbim_set_drops(self._h, n, P, lam, _ptr(xcoef), _stream()),
                    "shbim_set_drops")
        self.p = [int(p) for p in p_list]

    def sizes(self):
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        self._check(self._L.shbim_sizes(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
                    "shbim_sizes")
        return a.value, b.value, c.value

    def target_geometry(self, out):
        self._check(self._L.shbim_target_geometry(self._h, _ptr(out), _stream()),
                    "shbim_target_geometry")

    # ---------------------------------------------------------------- operators
    def sht(self, direction: int, grid: int, field_drop, inp, out):
        """shbim_sht: transform len(field_drop) fields, field f on drop field_drop[f]."""
        n = len(field_drop)
        fd = (ctypes.c_int32 * max(1, n))(*[int(d) for d in field_drop])
        self._check(self._L.shbim_sht(self._h, direction, grid, n, fd, _ptr(inp), _ptr(out), _stream()),
                    "shbim_sht")

    def eval_electric(self, which: int, dens, out, out_kind: int = OUT_COEF):
        self._check(self._L.shbim_eval_electric(self._h, which, _ptr(dens), _ptr(out), out_kind,
                                                _stream()), "shbim_eval_electric")

    def eval_stokes(self, f, u, out, out_kind: int = OUT_COEF):
        self._check(self._L.shbim_eval_stokes(self._h, _ptr(f), _ptr(u), _ptr(out), out_kind,
                                              _stream()), "shbim_eval_stokes")

    # ---------------------------------------------------------------- GMRES
    def gmres_begin(self, sys: int, rhs, x0=None):
        self._check(self._L.shbim_gmres_begin(self._h, sys, _ptr(rhs), _ptr(x0), _stream()),
                    "shbim_gmres_begin")

    def gmres_step(self):
        r = ctypes.c_double()
        rc = self._check(self._L.shbim_gmres_step(self._h, ctypes.byref(r), _stream()),
                         "shbim_gmres_step")
        return rc, r.value

    def gmres_finish(self, x):
        it = ctypes.c_int32()
        self._check(self._L.shbim_gmres_finish(self._h, _ptr(x), ctypes.byref(it), _stream()),
                    "shbim_gmres_finish")
        return it.value

    def gmres_solve(self, sys: int, rhs, x, x0=None):
        it = ctypes.c_int32()
        r = ctypes.c_double()
        self._check(self._L.shbim_gmres_solve(self._h, sys, _ptr(rhs), _ptr(x0), _ptr(x),
                                              ctypes.byref(it), ctypes.byref(r), _stream()),
                    "shbim_gmres_solve")
        return it.value, r.value

    def electric_rhs(self, E_u, out, E_q: float = 0.0):
        E = (ctypes.c_double * 3)(*[float(v) for v in E_u])
        self._check(self._L.shbim_electric_rhs(self._h, E, float(E_q), _ptr(out), _stream()),
                    "shbim_electric_rhs")

    def set_timing(self, on: bool):
        self._check(self._L.shbim_set_timing(self._h, 1 if on else 0), "shbim_set_timing")

    def kernel_work(self, cls: int) -> float:
        """Algorithmic flops of the bracketed launches of one class (shbim_kernel_work)."""
        w = ctypes.c_double()
        self._check(self._L.shbim_kernel_work(self._h, cls, ctypes.byref(w)), "shbim_kernel_work")
        return w.value

    def kernel_stats(self, cls: int):
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        self._check(self._L.shbim_kernel_stats(self._h, cls, ctypes.byref(ms), ctypes.byref(n)),
                    "shbim_kernel_stats")
        return ms.value, n.value

    def gmres_solve_refined(self, sys: int, rhs, x, x0=None, inner_tol: float = 1e-5,
                            max_outer: int = 10):
        inner = ctypes.c_int32()
        outer = ctypes.c_int32()
        r = ctypes.c_double()
        self._check(self._L.shbim_gmres_solve_refined(self._h, sys, _ptr(rhs), _ptr(x0), _ptr(x),
                                                      float(inner_tol), int(max_outer),
                                                      ctypes.byref(inner), ctypes.byref(outer),
                                                      ctypes.byref(r), _stream()),
                    "shbim_gmres_solve_refined")
        return inner.value, outer.value, r.value

    def rates(self, ph, gamma, u, gE):
        it = (ctypes.c_int32 * 2)()
        self._check(self._L.shbim_rates(self._h, ctypes.byref(ph), _ptr(gamma), _ptr(u), _ptr(gE), it,
                                        _stream()), "shbim_rates")
        return list(it)

    def step(self, ph, x, gamma, dt, x_out, gamma_out):
        err = ctypes.c_double()
        it = (ctypes.c_int32 * 4)()
        self._check(self._L.shbim_step(self._h, ctypes.byref(ph), _ptr(x), _ptr(gamma), float(dt),
                                       _ptr(x_out), _ptr(gamma_out), ctypes.byref(err), it, _stream()),
                    "shbim_step")
        return err.value, list(it)

    def reparametrize(self, x, gamma=None, steps: int = 20, a: float = 4.0, c: float = 0.5):
        """shbim_reparametrize: `steps` tangential flow steps on x (3 ncoef, in place) and gamma (ncoef, in place,
        or None); returns the energies before the first and after every step."""
        e = (ctypes.c_double * (int(steps) + 1))()
        self._check(self._L.shbim_reparametrize(self._h, int(steps), float(a), float(c), _ptr(x),
                                                None if gamma is None else _ptr(gamma), e, _stream()),
                    "shbim_reparametrize")
        return list(e)

    def stokes_rhs(self, ph, gamma, En, out):
        """shbim_stokes_rhs: -sum_j S_j[f/Ca_E - f^E] for the given E_n (3 ncoef coefficients into out)."""
        self._check(self._L.shbim_stokes_rhs(self._h, ctypes.byref(ph), _ptr(gamma), _ptr(En), _ptr(out), _stream()),
                    "shbim_stokes_rhs")

    def laplace_beltrami(self, coef, out):
        self._check(self._L.shbim_laplace_beltrami(self._h, _ptr(coef), _ptr(out), _stream()),
                    "shbim_laplace_beltrami")

    def set_field_shape(self, G):
        """shbim_set_field_shape: E_inf = E_u + E_q G x (G symmetric and traceless, 3 x 3)."""
        rows = [list(r) for r in G]
        if len(rows) != 3 or any(len(r) != 3 for r in rows):
            raise ValueError("field shape must be 3 x 3")
        g = (ctypes.c_double * 9)(*[float(v) for r in rows for v in r])
        self._check(self._L.shbim_set_field_shape(self._h, g), "shbim_set_field_shape")

    def set_stokes_preconditioner(self, on: bool):
        """shbim_set_stokes_preconditioner: right preconditioner of the Stokes system (rigid and normal modes)."""
        self._check(self._L.shbim_set_stokes_preconditioner(self._h, 1 if on else 0),
                    "shbim_set_stokes_preconditioner")

    def set_quantized_pairs(self, on: bool):
        """shbim_set_quantized_pairs: FP64-class pair sums on quantised positions (True) or general double-float."""
        self._check(self._L.shbim_set_quantized_pairs(self._h, 1 if on else 0), "shbim_set_quantized_pairs")

    def set_equation_of_state(self, law: int):
        """shbim_set_equation_of_state: EOS_LANGMUIR (beta, x_s) or EOS_LINEAR (gamma = 1 + beta (1 - Gamma))."""
        self._check(self._L.shbim_set_equation_of_state(self._h, int(law)), "shbim_set_equation_of_state")

    def set_diffusion(self, c: float):
        self._check(self._L.shbim_set_diffusion(self._h, float(c)), "shbim_set_diffusion")

    def set_outer_precision(self, precision: int):
        self._check(self._L.shbim_set_outer_precision(self._h, int(precision)), "shbim_set_outer_precision")

    def set_rows_precision(self, precision: int):
        self._check(self._L.shbim_set_rows_precision(self._h, int(precision)), "shbim_set_rows_precision")

    def set_oneshot_precision(self, precision: int):
        self._check(self._L.shbim_set_oneshot_precision(self._h, precision), "shbim_set_oneshot_precision")

    def set_self_precision(self, precision: int):
        self._check(self._L.shbim_set_self_precision(self._h, precision), "shbim_set_self_precision")

    def set_tensor_cores(self, on):
        """Tensor-core stages of the row build: True (the default set, TC_FOURIER | TC_ROTATION),
        False (none) or a mask of TC_FOURIER, TC_ROTATION and TC_LEGENDRE."""
        mask = ((TC_FOURIER | TC_ROTATION) if on else 0) if isinstance(on, bool) else int(on)
        self._check(self._L.shbim_set_tensor_cores(self._h, mask), "shbim_set_tensor_cores")

    def set_autotune(self, on: bool):
        self._check(self._L.shbim_set_autotune(self._h, 1 if on else 0), "shbim_set_autotune")

    def pair_shape(self, kind: int):
        """(targets per thread, source splits, fixed) of the FP32 pair kernel `kind`."""
        t = ctypes.c_int32()
        sp = ctypes.c_int32()
        rc = self._L.shbim_pair_shape(self._h, int(kind), ctypes.byref(t), ctypes.byref(sp))
        if rc < 0:
            self._check(rc, "shbim_pair_shape")
        return t.value, sp.value, rc == 1

    def set_pair_shape(self, kind: int, tpt: int, splits: int):
        self._check(self._L.shbim_set_pair_shape(self._h, int(kind), int(tpt), int(splits)),
                    "shbim_set_pair_shape")

    def pair_queue(self, kind: int) -> bool:
        """True when the FP32 pair kernel `kind` runs as persistent CTAs on a work counter."""
        rc = self._L.shbim_pair_queue(self._h, int(kind))
        if rc < 0:
            self._check(rc, "shbim_pair_queue")
        return rc == 1

    def set_pair_queue(self, kind: int, on: bool):
        self._check(self._L.shbim_set_pair_queue(self._h, int(kind), 1 if on else 0), "shbim_set_pair_queue")

    def set_device_gmres(self, on: bool):
        self._check(self._L.shbim_set_device_gmres(self._h, 1 if on else 0), "shbim_set_device_gmres")

    def set_graphs(self, on: bool):
        self._check(self._L.shbim_set_graphs(self._h, 1 if on else 0), "shbim_set_graphs")

    def set_concurrency(self, on: bool):
        """Run the self rows and near-field correction beside the all-pairs sums on a second
        library stream (on by default)."""
        self._check(self._L.shbim_set_concurrency(self._h, 1 if on else 0), "shbim_set_concurrency")

    def set_near(self, on: bool):
        self._check(self._L.shbim_set_near(self._h, 1 if on else 0), "shbim_set_near")

    def near_min_distance(self):
        """(smallest near-target distance to another drop's surface, the same in units of h_j)."""
        d, r = ctypes.c_double(), ctypes.c_double()
        self._check(self._L.shbim_near_min_distance(self._h, ctypes.byref(d), ctypes.byref(r)),
                    "shbim_near_min_distance")
        return d.value, r.value

    def set_wait_limit(self, seconds: float):
        self._check(self._L.shbim_set_wait_limit(self._h, float(seconds)), "shbim_set_wait_limit")

    def check_wait(self, arrive: bool) -> int:
        """shbim_check_wait: returns the library's status code (0, or SHBIM_ERR_TIMEOUT = -5)."""
        return int(self._L.shbim_check_wait(self._h, 1 if arrive else 0, _stream()))

    def warm_start_feature_count(self) -> int:
        return int(self._L.shbim_warm_start_feature_count(self._h))

    def warm_start_features(self, xcoef, gamma, ph, feat):
        """shbim_warm_start_features into a CUDA float32 tensor of warm_start_feature_count() values."""
        self._check(self._L.shbim_warm_start_features(self._h, _ptr(xcoef), _ptr(gamma), ctypes.byref(ph),
                                                      _ptr32(feat), _stream()), "shbim_warm_start_features")

    def learned_guess(self, net, feat, rhs_e=None, En0=None, u0=None):
        self._check(self._L.shbim_learned_guess(self._h, net._h, _ptr32(feat), _ptr(rhs_e), _ptr(En0), _ptr(u0),
                                                _stream()), "shbim_learned_guess")

    def set_warm_start(self, net):
        """Network used by rates() and step() for the initial guesses of both solves (None: none)."""
        self._check(self._L.shbim_set_warm_start(self._h, None if net is None else net._h), "shbim_set_warm_start")

    def near_pairs(self) -> int:
        return int(self._L.shbim_near_pairs(self._h))

    def operator_applications(self) -> int:
        return int(self._L.shbim_operator_applications(self._h))

    def launch_count(self) -> int:
        return int(self._L.shbim_launch_count(self._h))


def probe_peak(kind: int, iters: int = 20000):
    """Measured throughput of one SM pipe (shbim_probe_peak): (ops per second, ms)."""
    L = lib()
    r = ctypes.c_double()
    ms = ctypes.c_double()
    rc = L.shbim_probe_peak(int(kind), int(iters), ctypes.byref(r), ctypes.byref(ms), _stream())
    if rc != 0:
        raise ShbimError("shbim_probe_peak failed (%d)" % rc)
    return r.value, ms.value


class MLP:
    """shbim_mlp: the warm-start network (bfloat16 weights, FP32 accumulation)."""

    def __init__(self, widths, max_batch: int):
        L = lib()
        self._L = L
        self.widths = [int(w) for w in widths]
        arr = (ctypes.c_int32 * len(widths))(*self.widths)
        h = ctypes.c_void_p()
        rc = L.shbim_mlp_create(len(widths) - 1, arr, int(max_batch), ctypes.byref(h))
        if rc != 0:
            raise ShbimError("shbim_mlp_create failed (%d)" % rc)
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._L.shbim_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_layer(self, l: int, W, b):
        import numpy as np
        W = np.ascontiguousarray(W, dtype=np.float32)
        b = np.ascontiguousarray(b, dtype=np.float32)
        rc = self._L.shbim_mlp_set_layer(self._h, l, W.ctypes.data_as(ctypes.c_void_p),
                                          b.ctypes.data_as(ctypes.c_void_p))
        if rc != 0:
            raise ShbimError("shbim_mlp_set_layer failed (%d)" % rc)

    def set_input_affine(self, shift, scale):
        import numpy as np
        if shift is None:
            rc = self._L.shbim_mlp_set_input_affine(self._h, None, None)
        else:
            a = np.ascontiguousarray(shift, dtype=np.float32)
            b = np.ascontiguousarray(scale, dtype=np.float32)
            rc = self._L.shbim_mlp_set_input_affine(self._h, a.ctypes.data_as(ctypes.c_void_p),
                                                     b.ctypes.data_as(ctypes.c_void_p))
        if rc != 0:
            raise ShbimError("shbim_mlp_set_input_affine failed (%d)" % rc)

    def get_layer(self, l: int):
        import numpy as np
        a, b = self.widths[l], self.widths[l + 1]
        W, bb = np.empty((b, a), np.float32), np.empty(b, np.float32)
        gW, gb = np.empty((b, a), np.float32), np.empty(b, np.float32)
        rc = self._L.shbim_mlp_get_layer(self._h, l, *(x.ctypes.data_as(ctypes.c_void_p) for x in (W, bb, gW, gb)))
        if rc != 0:
            raise ShbimError("shbim_mlp_get_layer failed (%d)" % rc)
        return W, bb, gW, gb

    def forward(self, x, y):
        rc = self._L.shbim_mlp_forward(self._h, x.shape[0], _ptr32(x), _ptr32(y), _stream())
        if rc != 0:
            raise ShbimError("shbim_mlp_forward failed (%d)" % rc)

    def train_step(self, x, t, lr: float, update: bool = True) -> float:
        loss = ctypes.c_double()
        rc = self._L.shbim_mlp_train_step(self._h, x.shape[0], _ptr32(x), _ptr32(t), float(lr),
                                           1 if update else 0, ctypes.byref(loss), _stream())
        if rc != 0:
            raise ShbimError("shbim_mlp_train_step failed (%d)" % rc)
        return loss.value


def electric_warm_start(ctx: Context, net: MLP, xcoef, rhs, x0):
    ctx._check(ctx._L.shbim_electric_warm_start(ctx._h, net._h, _ptr(xcoef), _ptr(rhs), _ptr(x0), _stream()),
               "shbim_electric_warm_start")
