"""Thin Python binding of liblsgpu.so (C ABI in include/lsgpu.h).

Argument marshalling only: every step of the solver runs in the library's CUDA
kernels (and its host setup).  Host arrays are numpy; device arrays are torch
CUDA tensors of dtype complex128 (PyTorch is used for device memory and
streams only).  Importing fails loudly when the library has not been built.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblsgpu.so")

LS_OK, LS_EINVAL, LS_ENOMEM, LS_ECUDA, LS_ESINGULAR, LS_ENOCONV, LS_ETIMEOUT = range(7)
_STATUS = {0: "LS_OK", 1: "LS_EINVAL", 2: "LS_ENOMEM", 3: "LS_ECUDA", 4: "LS_ESINGULAR", 5: "LS_ENOCONV",
           6: "LS_ETIMEOUT"}

EXPORTED = ["ls_params_default", "ls_mesh_create", "ls_mesh_destroy", "ls_mesh_num_nodes", "ls_operator_create",
            "ls_cartesian_create",
            "ls_op_destroy", "ls_op_num_nodes", "ls_apply_dev", "ls_apply", "ls_apply_precond_dev",
            "ls_apply_precond_batch_dev", "ls_pairsum_dev",
            "ls_solve", "ls_solve_dev", "ls_op_correction", "ls_correction_host", "ls_correction_dev", "ls_grid_host", "ls_transfer_host",
            "ls_hankel0_dev",
            "ls_pairsum_batch_dev", "ls_solve_batch_dev", "ls_solve_multi_dev", "ls_apply_transpose_dev", "ls_potential_transpose_dev", "ls_apply_precond_transpose_dev",
            "ls_solve_transpose_dev", "ls_op_set_contrast", "ls_incident_dev", "ls_misfit_gradient_dev",
            "ls_solve_transpose_batch_dev", "ls_misfit_gradient_batch_dev",
            "ls_op_set_batch_kernel", "ls_op_set_batch_refine", "ls_op_set_stall_test", "ls_tc_gemm_check",
            "ls_apply_precond", "ls_apply_transpose", "ls_solve_adjoint", "ls_residual_dev", "ls_op_last_residual",
            "ls_op_set_contrast_dev", "ls_misfit_dev", "ls_op_ritz", "ls_hessenberg_eigenvalues",
            "ls_precond_rho_dev",
            "ls_op_set_pairsum", "ls_op_set_pair_symmetry", "ls_op_set_timing", "ls_op_setup_times", "ls_op_tuning", "ls_op_stats", "ls_op_stats_kind", "ls_probe_fp64", "ls_pairsum_noalloc", "ls_last_error"]


class LsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


LS_PREC_FP64_TABLE, LS_PREC_FP64_DIRECT, LS_PREC_FP32, LS_PREC_FP64_DF, LS_PREC_MIXED = range(5)


class Params(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("use_precond", ctypes.c_int32),
                ("kappa", ctypes.c_double), ("box", ctypes.c_double * 4), ("nx", ctypes.c_int32),
                ("ny", ctypes.c_int32), ("prec", ctypes.c_int32), ("approach", ctypes.c_int32),
                ("setup_on_device", ctypes.c_int32)]

    @property
    def pairsum(self):
        """The pair-sum arithmetic (alias of prec)."""
        return self.prec

    @pairsum.setter
    def pairsum(self, v):
        self.prec = v


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing; build it with `python paper_2608_17615_b300/build.py`")
    lib = ctypes.CDLL(LIB_PATH)
    P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "ls_params_default": (None, [P]),
        "ls_mesh_create": (I32, [I32, P, I32, P, P, P, P, I32, P, P, P, P]),
        "ls_mesh_destroy": (None, [P]),
        "ls_mesh_num_nodes": (I32, [P]),
        "ls_operator_create": (I32, [P, D, P, P, P, P, P]),
        "ls_cartesian_create": (I32, [D, P, P, P, P]),
        "ls_op_destroy": (None, [P]),
        "ls_op_num_nodes": (I32, [P]),
        "ls_apply_dev": (I32, [P, P, P]),
        "ls_apply": (I32, [P, P, P]),
        "ls_apply_precond_dev": (I32, [P, P, P]),
        "ls_apply_precond_batch_dev": (I32, [P, I32, P, P]),
        "ls_pairsum_dev": (I32, [P, P, P]),
        "ls_solve": (I32, [P, I32, P, P, I32, P, P, P, P, P]),
        "ls_apply_precond": (I32, [P, P, P]),
        "ls_apply_transpose": (I32, [P, P, P]),
        "ls_solve_adjoint": (I32, [P, I32, P, P, P]),
        "ls_residual_dev": (I32, [P, P, P, P]),
        "ls_op_last_residual": (I32, [P, P]),
        "ls_op_set_contrast_dev": (I32, [P, P, I32]),
        "ls_misfit_dev": (I32, [P, I32, P, P, P, P]),
        "ls_op_ritz": (I32, [P, I32, P, P]),
        "ls_precond_rho_dev": (I32, [P, I32, P, P]),
        "ls_hessenberg_eigenvalues": (I32, [I32, P, P]),
        "ls_solve_dev": (I32, [P, I32, P, P, I32, P, P, P]),
        "ls_op_correction": (I32, [P, P, P, P, P]),
        "ls_correction_host": (I32, [P, D, D, P, P, P, P]),
        "ls_correction_dev": (I32, [P, D, D, P, P, P, P, P, P]),
        "ls_transfer_host": (I32, [P, P, I32, I32, I32, P, P, P, P, P]),
        "ls_grid_host": (I32, [P, D, P, I32, I32, P, P, P]),
        "ls_hankel0_dev": (I32, [I64, P, P, P]),
        "ls_pairsum_batch_dev": (I32, [P, I32, P, P]),
        "ls_solve_batch_dev": (I32, [P, I32, P, P, I32, P, P, P]),
        "ls_solve_multi_dev": (I32, [I32, P, I32, P, P, P]),
        "ls_apply_transpose_dev": (I32, [P, P, P]),
        "ls_potential_transpose_dev": (I32, [P, P, P]),
        "ls_apply_precond_transpose_dev": (I32, [P, P, P]),
        "ls_solve_transpose_dev": (I32, [P, I32, P, P, P]),
        "ls_op_set_contrast": (I32, [P, P]),
        "ls_incident_dev": (I32, [P, I32, P, P]),
        "ls_misfit_gradient_dev": (I32, [P, I32, P, I32, P, P, P, P]),
        "ls_solve_transpose_batch_dev": (I32, [P, I32, P, P, P]),
        "ls_op_set_batch_kernel": (I32, [P, I32, I32, I32]),
        "ls_op_set_batch_refine": (I32, [P, I32]),
        "ls_op_set_stall_test": (I32, [P, D]),
        "ls_tc_gemm_check": (I32, [I32, P]),
        "ls_misfit_gradient_batch_dev": (I32, [P, I32, P, I32, P, P, P, P]),
        "ls_op_set_pairsum": (I32, [P, I32]),
        "ls_op_set_pair_symmetry": (I32, [P, I32]),
        "ls_op_set_timing": (I32, [P, I32]),
        "ls_op_setup_times": (I32, [P, P]),
        "ls_op_tuning": (I32, [P, P, P, P]),
        "ls_op_stats": (I32, [P, P, P, P]),
        "ls_op_stats_kind": (I32, [P, I32, P, P]),
        "ls_probe_fp64": (I32, [P, P]),
        "ls_pairsum_noalloc": (I32, [I32, P, P, P, D, P, P]),
        "ls_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


def last_error():
    return _lib.ls_last_error().decode()


def _check(status, allow=()):
    if status != LS_OK and status not in allow:
        raise LsError(status, last_error())
    return status


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _dptr(t):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("device arguments must be contiguous CUDA tensors")
    return ctypes.c_void_p(t.data_ptr())


def _c128(a):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a, a.view(np.float64)


def params_default():
    p = Params()
    _lib.ls_params_default(ctypes.byref(p))
    return p


class Mesh:
    """ls_mesh handle built from an lsinput.mesh.Mesh-like object."""

    def __init__(self, m):
        self._keep = [np.ascontiguousarray(m.vertices, np.float64), np.ascontiguousarray(m.tris, np.int32),
                      np.ascontiguousarray(m.domain, np.int32), np.ascontiguousarray(m.edge_curve, np.int32),
                      np.ascontiguousarray(m.edge_theta, np.float64), np.ascontiguousarray(m.curves, np.float64),
                      np.ascontiguousarray(m.nodes, np.float64), np.ascontiguousarray(m.weights, np.float64)]
        v, t, d, ec, et, cu, nd, w = self._keep
        h = ctypes.c_void_p()
        _check(_lib.ls_mesh_create(v.shape[0], _ptr(v), t.shape[0], _ptr(t), _ptr(d), _ptr(ec), _ptr(et),
                                   cu.shape[0], _ptr(cu), _ptr(nd), _ptr(w), ctypes.byref(h)))
        self.handle = h
        self.n = _lib.ls_mesh_num_nodes(h)

    def __del__(self):
        if getattr(self, "handle", None):
            _lib.ls_mesh_destroy(self.handle)
            self.handle = None


class Operator:
    """ls_op handle: L = I + k^2 V M and optionally the preconditioner P."""

    def __init__(self, mesh, k, m, m_grid=None, params=None, stream=None, **overrides):
        p = params if params is not None else params_default()
        for key, val in overrides.items():
            if key == "box":
                for i in range(4):
                    p.box[i] = val[i]
            elif key == "pairsum":
                p.prec = val
            else:
                if key not in dict(Params._fields_):
                    raise TypeError(f"unknown operator parameter {key!r}")
                setattr(p, key, val)
        self.params = p
        m_arr, m_f = _c128(m)
        mg_f = None
        if m_grid is not None:
            self._mg, mg_f = _c128(m_grid)
        h = ctypes.c_void_p()
        if stream is None:
            stream = _current_stream()
        _check(_lib.ls_operator_create(mesh.handle, float(k), _ptr(m_f), _ptr(mg_f), ctypes.byref(p),
                                       ctypes.c_void_p(stream), ctypes.byref(h)))
        self.handle = h
        self.n = _lib.ls_op_num_nodes(h)
        self.k = float(k)

    def __del__(self):
        if getattr(self, "handle", None):
            _lib.ls_op_destroy(self.handle)
            self.handle = None

    def apply_dev(self, x, y):
        _check(_lib.ls_apply_dev(self.handle, _dptr(x), _dptr(y)))

    def apply(self, x):
        x, xf = _c128(x)
        y = np.empty_like(x)
        _check(_lib.ls_apply(self.handle, _ptr(xf), _ptr(y.view(np.float64))))
        return y

    def apply_precond(self, x):
        """y = P x with host buffers."""
        x, xf = _c128(x)
        y = np.empty_like(x)
        _check(_lib.ls_apply_precond(self.handle, _ptr(xf), _ptr(y.view(np.float64))))
        return y

    def apply_transpose(self, x):
        """y = L^T x with host buffers."""
        x, xf = _c128(x)
        y = np.empty_like(x)
        _check(_lib.ls_apply_transpose(self.handle, _ptr(xf), _ptr(y.view(np.float64))))
        return y

    def solve_adjoint(self, g):
        """L^T lambda = g for host g [R, N]; returns (lambda [R, N], iters [R], status)."""
        g, gf = _c128(np.atleast_2d(g))
        lam = np.empty_like(g)
        iters = np.zeros(g.shape[0], np.int32)
        st = _check(_lib.ls_solve_adjoint(self.handle, g.shape[0], _ptr(gf), _ptr(lam.view(np.float64)), _ptr(iters)),
                    allow=(LS_ENOCONV,))
        return lam, iters, st

    def residual_dev(self, b, u):
        """||P (b - L u)|| / ||P b|| by full applies (device tensors of N complex)."""
        r = ctypes.c_double()
        _check(_lib.ls_residual_dev(self.handle, _dptr(b), _dptr(u), ctypes.byref(r)))
        return r.value

    def ritz(self):
        """Ritz values (eigenvalues of the square Hessenberg matrix) of the last single-system solve."""
        cnt = ctypes.c_int32()
        _check(_lib.ls_op_ritz(self.handle, 0, ctypes.byref(cnt), None))
        out = np.empty(cnt.value, np.complex128)
        if cnt.value:
            _check(_lib.ls_op_ritz(self.handle, cnt.value, ctypes.byref(cnt), _ptr(out.view(np.float64))))
        return out

    def precond_rho_dev(self, X):
        """rho(R_II x) (Eq. rho_def) for grid vectors X torch [R, nx * ny] complex128; numpy [R] complex."""
        R = X.shape[0]
        out = np.empty(R, np.complex128)
        _check(_lib.ls_precond_rho_dev(self.handle, R, _dptr(X), _ptr(out.view(np.float64))))
        return out

    def last_residual(self):
        """Largest explicit GMRES exit residual of the last single-system solve call."""
        r = ctypes.c_double()
        _check(_lib.ls_op_last_residual(self.handle, ctypes.byref(r)))
        return r.value

    def set_contrast_dev(self, m):
        """Contrast from a device tensor: [N] complex128, or [N] float64 (real part)."""
        import torch
        if m.dtype == torch.float64:
            _check(_lib.ls_op_set_contrast_dev(self.handle, _dptr(m), 1))
        elif m.dtype == torch.complex128:
            _check(_lib.ls_op_set_contrast_dev(self.handle, _dptr(m), 0))
        else:
            raise ValueError("contrast must be float64 or complex128")

    def misfit_dev(self, uinf, target, resid):
        """resid = uinf - target and J = 1/2 sum |resid|^2 on device tensors; returns J."""
        J = ctypes.c_double()
        _check(_lib.ls_misfit_dev(self.handle, int(uinf.numel()), _dptr(uinf), _dptr(target), _dptr(resid),
                                  ctypes.byref(J)))
        return J.value

    def apply_precond_dev(self, x, y):
        _check(_lib.ls_apply_precond_dev(self.handle, _dptr(x), _dptr(y)))

    def apply_precond_batch_dev(self, x, y):
        """y_r = P x_r for device tensors x, y [R, N] with the batched kernels."""
        _check(_lib.ls_apply_precond_batch_dev(self.handle, x.shape[0], _dptr(x), _dptr(y)))

    def pairsum_dev(self, f, y):
        _check(_lib.ls_pairsum_dev(self.handle, _dptr(f), _dptr(y)))

    def solve(self, dir_angles=None, ff_angles=None, want_u=True, want_hist=True, b=None):
        """Host-buffer solve for plane waves (dir_angles) or explicit right-hand sides b [R, N];
        returns (u [R, N], uinf [R, n_ff], hist [R, max_iter+1], iters [R], status)."""
        bf = None
        if b is not None:
            b, bf = _c128(np.atleast_2d(b))
            R = b.shape[0]
            dirs = None
        else:
            dirs = np.ascontiguousarray(dir_angles, np.float64).ravel()
            R = dirs.size
        ff = np.ascontiguousarray(ff_angles if ff_angles is not None else [], np.float64).ravel()
        u = np.empty((R, self.n), np.complex128) if want_u else None
        uinf = np.empty((R, ff.size), np.complex128) if ff.size else None
        hist = np.zeros((R, self.params.max_iter + 1)) if want_hist else None
        iters = np.zeros(R, np.int32)
        st = _check(_lib.ls_solve(self.handle, R, _ptr(dirs), _ptr(bf), ff.size, _ptr(ff) if ff.size else None,
                                  _ptr(u.view(np.float64)) if u is not None else None,
                                  _ptr(uinf.view(np.float64)) if uinf is not None else None,
                                  _ptr(hist), _ptr(iters)), allow=(LS_ENOCONV,))
        return u, uinf, hist, iters, st

    def solve_dev(self, b, u, ff_angles=None, uinf=None):
        """Device-buffer solve: b, u torch [R, N] complex128; uinf torch [R, n_ff] or None."""
        R = b.shape[0] if b.dim() == 2 else 1
        ff = np.ascontiguousarray(ff_angles if ff_angles is not None else [], np.float64).ravel()
        iters = np.zeros(R, np.int32)
        st = _check(_lib.ls_solve_dev(self.handle, R, _dptr(b), _dptr(u), ff.size, _ptr(ff) if ff.size else None,
                                      _dptr(uinf), _ptr(iters)), allow=(LS_ENOCONV,))
        return iters, st

    def pairsum_batch_dev(self, f, y):
        """Batched naive pair sum for f, y torch [R, N] complex128."""
        _check(_lib.ls_pairsum_batch_dev(self.handle, f.shape[0], _dptr(f), _dptr(y)))

    def solve_batch_dev(self, b, u, ff_angles=None, uinf=None):
        """R lock-step solves: b, u torch [R, N]; uinf torch [R, n_ff] or None."""
        R = b.shape[0]
        ff = np.ascontiguousarray(ff_angles if ff_angles is not None else [], np.float64).ravel()
        iters = np.zeros(R, np.int32)
        st = _check(_lib.ls_solve_batch_dev(self.handle, R, _dptr(b), _dptr(u), ff.size, _ptr(ff) if ff.size else None,
                                            _dptr(uinf), _ptr(iters)), allow=(LS_ENOCONV,))
        return iters, st

    def apply_transpose_dev(self, x, y):
        _check(_lib.ls_apply_transpose_dev(self.handle, _dptr(x), _dptr(y)))

    def potential_transpose_dev(self, x, y):
        _check(_lib.ls_potential_transpose_dev(self.handle, _dptr(x), _dptr(y)))

    def apply_precond_transpose_dev(self, x, y):
        _check(_lib.ls_apply_precond_transpose_dev(self.handle, _dptr(x), _dptr(y)))

    def solve_transpose_dev(self, g, lam):
        R = g.shape[0] if g.dim() == 2 else 1
        iters = np.zeros(R, np.int32)
        st = _check(_lib.ls_solve_transpose_dev(self.handle, R, _dptr(g), _dptr(lam), _ptr(iters)), allow=(LS_ENOCONV,))
        return iters, st

    def set_contrast(self, m):
        m, mf = _c128(m)
        _check(_lib.ls_op_set_contrast(self.handle, _ptr(mf)))

    def incident_dev(self, dir_angles, b):
        dirs = np.ascontiguousarray(dir_angles, np.float64).ravel()
        _check(_lib.ls_incident_dev(self.handle, dirs.size, _ptr(dirs), _dptr(b)))

    def misfit_gradient_dev(self, u, ff_angles, resid, grad):
        """grad [N] float64 tensor <- dJ/dRe(m); u [R, N], resid [R, n_ff] complex128 tensors."""
        ff = np.ascontiguousarray(ff_angles, np.float64).ravel()
        R = u.shape[0] if u.dim() == 2 else 1
        iters = np.zeros(R, np.int32)
        st = _check(_lib.ls_misfit_gradient_dev(self.handle, R, _dptr(u), ff.size, _ptr(ff), _dptr(resid),
                                                _dptr(grad), _ptr(iters)), allow=(LS_ENOCONV,))
        return iters, st

    def solve_transpose_batch_dev(self, g, lam):
        R = g.shape[0]
        iters = np.zeros(R, np.int32)
        st = _check(_lib.ls_solve_transpose_batch_dev(self.handle, R, _dptr(g), _dptr(lam), _ptr(iters)),
                    allow=(LS_ENOCONV,))
        return iters, st

    def misfit_gradient_batch_dev(self, u, ff_angles, resid, grad):
        ff = np.ascontiguousarray(ff_angles, np.float64).ravel()
        R = u.shape[0]
        iters = np.zeros(R, np.int32)
        st = _check(_lib.ls_misfit_gradient_batch_dev(self.handle, R, _dptr(u), ff.size, _ptr(ff), _dptr(resid),
                                                      _dptr(grad), _ptr(iters)), allow=(LS_ENOCONV,))
        return iters, st

    def set_pairsum(self, mode):
        """LS_PREC_*: 0 FP64 table, 1 FP64 direct, 2 FP32, 3 double-float, 4 mixed."""
        _check(_lib.ls_op_set_pairsum(self.handle, int(mode)))
        self.params.prec = int(mode)

    def set_pair_symmetry(self, on):
        """Double-float pair sum over unordered pairs (True, default) or every ordered pair."""
        _check(_lib.ls_op_set_pair_symmetry(self.handle, int(bool(on))))

    def set_batch_refine(self, accurate):
        """Refinement residuals of the batched solves from the single-RHS pair sum (True) or
        the batched FP32 operator (False, default)."""
        _check(_lib.ls_op_set_batch_refine(self.handle, int(bool(accurate))))

    def set_batch_kernel(self, kind, fold=4, refine=4):
        """Batched pair sum on 0: CUDA cores (FP32), 1: tensor cores (accumulator restarted every
        fold stages; batched solves refined up to `refine` times), 2: CUDA cores in double-float
        (FP64-accurate; operators built with the double-float or mixed form)."""
        _check(_lib.ls_op_set_batch_kernel(self.handle, int(kind), int(fold), int(refine)))

    def set_stall_test(self, stall_ms):
        """Failure-detection test: the next tensor-core launches stall stall_ms on a
        barrier nothing completes and return LS_ETIMEOUT (0 turns it off)."""
        _check(_lib.ls_op_set_stall_test(self.handle, float(stall_ms)))

    def set_timing(self, on=True):
        _check(_lib.ls_op_set_timing(self.handle, 1 if on else 0))

    def setup_times(self):
        """(correction, grid, block LU, table) setup wall times in seconds."""
        t = np.zeros(4)
        _check(_lib.ls_op_setup_times(self.handle, _ptr(t)))
        return tuple(t)

    def tuning(self):
        """(table coefficients per cell in use, timed ms of the 12/10/9/8-coefficient candidates)."""
        nc = ctypes.c_int32()
        ms = np.zeros(4)
        _check(_lib.ls_op_tuning(self.handle, ctypes.byref(nc), _ptr(ms), None))
        return nc.value, tuple(ms)

    def df_tail(self):
        """Double-float form: Horner coefficients summed in plain FP32 (per chain)."""
        nf = ctypes.c_int32()
        _check(_lib.ls_op_tuning(self.handle, None, None, ctypes.byref(nf)))
        return nf.value

    def stats(self):
        """(pair-sum kernel ms, pair-sum launches, kernel launches) since the last set_timing."""
        ms = ctypes.c_double()
        pl = ctypes.c_int64()
        la = ctypes.c_int64()
        _check(_lib.ls_op_stats(self.handle, ctypes.byref(ms), ctypes.byref(pl), ctypes.byref(la)))
        return ms.value, pl.value, la.value

    def stats_kind(self, kind):
        """(ms, launches) of the timed pair-sum launches of one arithmetic (LS_PREC_*; 10, 11:
        the CUDA-core and tensor-core batched kernels)."""
        ms = ctypes.c_double()
        pl = ctypes.c_int64()
        _check(_lib.ls_op_stats_kind(self.handle, int(kind), ctypes.byref(ms), ctypes.byref(pl)))
        return ms.value, pl.value

    def correction(self):
        """The library's correction dV as (rowptr, cols, vals)."""
        nnz = ctypes.c_int64()
        _check(_lib.ls_op_correction(self.handle, ctypes.byref(nnz), None, None, None))
        rp = np.empty(self.n + 1, np.int64)
        ci = np.empty(nnz.value, np.int32)
        va = np.empty(nnz.value, np.complex128)
        _check(_lib.ls_op_correction(self.handle, ctypes.byref(nnz), _ptr(rp), _ptr(ci), _ptr(va.view(np.float64))))
        return rp, ci, va


class CartesianOperator(Operator):
    """Purely Cartesian L^(C) on the grid of box / nx / ny (ls_cartesian_create): unknowns
    at the grid nodes, preconditioner S^(C) when use_precond."""

    def __init__(self, k, m_grid, params=None, stream=None, **overrides):
        p = params if params is not None else params_default()
        for key, val in overrides.items():
            if key == "box":
                for i in range(4):
                    p.box[i] = val[i]
            else:
                if key not in dict(Params._fields_):
                    raise TypeError(f"unknown operator parameter {key!r}")
                setattr(p, key, val)
        self.params = p
        _, mg = _c128(m_grid)
        h = ctypes.c_void_p()
        if stream is None:
            stream = _current_stream()
        _check(_lib.ls_cartesian_create(float(k), _ptr(mg), ctypes.byref(p), ctypes.c_void_p(stream), ctypes.byref(h)))
        self.handle = h
        self.n = _lib.ls_op_num_nodes(h)
        self.k = float(k)


def hessenberg_eigenvalues(H):
    """Eigenvalues of an upper Hessenberg matrix (host routine of the Ritz values)."""
    H = np.asfortranarray(np.asarray(H, np.complex128))
    n = H.shape[0]
    e = np.empty(n, np.complex128)
    _check(_lib.ls_hessenberg_eigenvalues(n, _ptr(H.ravel(order="F").view(np.float64)), _ptr(e.view(np.float64))))
    return e


def correction_host(mesh, k, kappa=3.0):
    """Host-only build of dV for a Mesh handle: (rowptr, cols, vals)."""
    nnz = ctypes.c_int64()
    _check(_lib.ls_correction_host(mesh.handle, float(k), float(kappa), ctypes.byref(nnz), None, None, None))
    rp = np.empty(mesh.n + 1, np.int64)
    ci = np.empty(nnz.value, np.int32)
    va = np.empty(nnz.value, np.complex128)
    _check(_lib.ls_correction_host(mesh.handle, float(k), float(kappa), ctypes.byref(nnz), _ptr(rp), _ptr(ci),
                                   _ptr(va.view(np.float64))))
    return rp, ci, va


def correction_dev(mesh, k, kappa=3.0):
    """Device build of dV for a Mesh handle: (rowptr, cols, vals, blocks rebuilt on the host)."""
    nnz = ctypes.c_int64()
    nh = ctypes.c_int64()
    st = ctypes.c_void_p(_current_stream())
    _check(_lib.ls_correction_dev(mesh.handle, float(k), float(kappa), st, ctypes.byref(nnz), None, None, None, None))
    rp = np.empty(mesh.n + 1, np.int64)
    ci = np.empty(nnz.value, np.int32)
    va = np.empty(nnz.value, np.complex128)
    _check(_lib.ls_correction_dev(mesh.handle, float(k), float(kappa), st, ctypes.byref(nnz), _ptr(rp), _ptr(ci),
                                  _ptr(va.view(np.float64)), ctypes.byref(nh)))
    return rp, ci, va, nh.value


def transfer_host(mesh, box, nx, ny, approach=2):
    """Host-only T_Q^C as (rowptr [nx*ny+1], cols, vals, interior count)."""
    bx = np.ascontiguousarray(box, np.float64)
    nnz = ctypes.c_int64()
    ni = ctypes.c_int32()
    _check(_lib.ls_transfer_host(mesh.handle, _ptr(bx), int(nx), int(ny), int(approach), ctypes.byref(nnz), None,
                                 None, None, None))
    rp = np.empty(nx * ny + 1, np.int64)
    ci = np.empty(nnz.value, np.int32)
    va = np.empty(nnz.value, np.float64)
    _check(_lib.ls_transfer_host(mesh.handle, _ptr(bx), int(nx), int(ny), int(approach), ctypes.byref(nnz), _ptr(rp),
                                 _ptr(ci), _ptr(va), ctypes.byref(ni)))
    return rp, ci, va, ni.value


def grid_host(mesh, k, box, nx, ny, m_grid):
    """Host-only preconditioner setup: (stencils [9 classes, 9 offsets], cband [ny, 3, 3, nx]) complex."""
    bx = np.ascontiguousarray(box, np.float64)
    mg = np.ascontiguousarray(np.asarray(m_grid, np.complex128).ravel())
    st = np.zeros((9, 9), np.complex128)
    cb = np.zeros((ny, 3, 3, nx), np.complex128)
    _check(_lib.ls_grid_host(mesh.handle, float(k), _ptr(bx), int(nx), int(ny), _ptr(mg.view(np.float64)),
                             _ptr(st.view(np.float64)), _ptr(cb.view(np.float64))))
    return st, cb


def solve_multi_dev(ops, B, U):
    """Several operators in lock step: B[s], U[s] torch [R, N_s] complex128.  Returns iters [S, R], status."""
    S = len(ops)
    R = B[0].shape[0]
    hs = (ctypes.c_void_p * S)(*[o.handle.value for o in ops])
    bs = (ctypes.c_void_p * S)(*[b.data_ptr() for b in B])
    us = (ctypes.c_void_p * S)(*[u.data_ptr() for u in U])
    iters = np.zeros((S, R), np.int32)
    st = _check(_lib.ls_solve_multi_dev(S, hs, R, bs, us, _ptr(iters)), allow=(LS_ENOCONV,))
    return iters, st


def hankel0_dev(z, out):
    """out[i] = H0^(1)(z[i]) by the device routine of the pair sum (z float64, out complex128 tensors)."""
    _check(_lib.ls_hankel0_dev(z.numel(), _dptr(z), _dptr(out), ctypes.c_void_p(_current_stream())))


def tc_gemm_check(N=128):
    """Max abs error of one exact 128 x N x 32 product through the tensor-core path (0 when right)."""
    e = ctypes.c_double()
    _check(_lib.ls_tc_gemm_check(int(N), ctypes.byref(e)))
    return e.value


def probe_fp64():
    """Measured FP64 FMA throughput of the current device, GFLOP/s."""
    g = ctypes.c_double()
    _check(_lib.ls_probe_fp64(ctypes.byref(g), ctypes.c_void_p(_current_stream())))
    return g.value


def pairsum_noalloc(xy, w, f, k, y):
    """Allocation-free pair sum on device tensors: xy [n, 2] and w [n] float64,
    f and y [n] complex128 (see ls_pairsum_noalloc for whom it serves).  The
    shapes and dtypes are checked here because the C call sees only pointers."""
    import torch
    n = int(f.numel())
    for name, t, dt in (("xy", xy, torch.float64), ("w", w, torch.float64), ("f", f, torch.complex128),
                        ("y", y, torch.complex128)):
        if not t.is_cuda or not t.is_contiguous() or t.dtype != dt:
            raise ValueError(f"{name} must be a contiguous CUDA tensor of dtype {dt}")
    if tuple(xy.shape) != (n, 2) or w.numel() != n or y.numel() != n:
        raise ValueError(f"shapes must be xy [{n}, 2], w [{n}], y [{n}]")
    _check(_lib.ls_pairsum_noalloc(n, _dptr(xy), _dptr(w), _dptr(f), float(k), _dptr(y),
                                   ctypes.c_void_p(_current_stream())))


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return 0
