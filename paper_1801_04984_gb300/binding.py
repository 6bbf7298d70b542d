"""Thin ctypes binding of the C ABI in include/biot.h.

Only argument marshalling happens here: every step of the computation runs in
the CUDA library (libbiot_gb300.so, built in-tree by `build.py`).  PyTorch
provides device memory and the current stream.  There is no CPU fallback: if
the library is missing, loading fails with an error.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbiot_gb300.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "biot.h")

OK, EINVAL, ENOMEM, ECUDA, ENOCONV, EBREAKDOWN, ETIMEOUT = range(7)
U_NATURAL, U_DIRICHLET, U_ROLLER = 0, 1, 2
F_NATURAL, F_NOFLOW = 0, 1
FP64, FP32, MIXED, FIXED_STRESS = 0, 1, 2, 3
LOAD_TRACTION_TOP, LOAD_MMS2D_CONST, LOAD_MMS2D_LINEAR = 0, 1, 2
PART_FLUX_MASS_INV, PART_SCHUR, PART_VCYCLE, PART_ELASTICITY, PART_SCHUR_STEP = 0, 1, 2, 3, 4
KERNEL_ELASTICITY_FP32, KERNEL_ELASTICITY_FP64, KERNEL_SCHUR_FP32, KERNEL_ELASTICITY_FP32_COARSE = 0, 1, 2, 3
ERR_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOCONV", 5: "EBREAKDOWN", 6: "ETIMEOUT"}


class Mesh(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("u_bc", C.c_int * 6), ("f_bc", C.c_int * 6)]


class Coeffs(C.Structure):
    _fields_ = [("b", C.c_double), ("invM", C.c_double), ("K_dr", C.c_double), ("lam", C.c_double),
                ("mu", C.c_double), ("eta", C.c_double), ("K_cell", C.POINTER(C.c_double))]


class Opts(C.Structure):
    _fields_ = [("gmres_restart", C.c_int), ("cheb_degree", C.c_int), ("schur_degree", C.c_int),
                ("mg_min_cells", C.c_int), ("beta_fs", C.c_double), ("flux_mass_exact", C.c_int), ("pair_coupling", C.c_int),
                ("schur_mg", C.c_int)]


class SolveOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iters", C.c_int), ("mode", C.c_int), ("inner_tol", C.c_double),
                ("transpose", C.c_int)]


class BatchItem(C.Structure):
    _fields_ = [("mesh", Mesh), ("coeffs", Coeffs), ("r", C.c_int), ("T", C.c_double), ("slabs", C.c_int),
                ("load_kind", C.c_int), ("load_value", C.c_double), ("nterms", C.c_int),
                ("f_terms", C.c_void_p), ("tcoef", C.c_void_p), ("U0", C.c_void_p), ("U_end", C.c_void_p)]


class Stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("refinements", C.c_int), ("restarts", C.c_int),
                ("rel_residual", C.c_double), ("seconds", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def header_functions():
    """Names of the functions declared in include/biot.h."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"\b(biot_[a-z_]+)\s*\(", txt)))


def load(path: str = LIB_PATH):
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("CUDA library %s not built (run paper_1801_04984_gb300.build.build())" % path)
    lib = C.CDLL(path)
    vp, dp, ip, i64p = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_int64)
    sig = {
        "biot_setup": (C.c_int, [C.POINTER(Mesh), C.POINTER(Coeffs), C.c_int, C.POINTER(Opts), C.POINTER(vp)]),
        "biot_setup_batch": (C.c_int, [C.POINTER(Mesh), C.POINTER(Coeffs), C.c_int, C.POINTER(Opts), C.c_int,
                                       C.POINTER(vp)]),
        "biot_march_batch": (C.c_int, [vp, C.c_double, C.c_int, C.c_int, C.POINTER(vp), dp, C.POINTER(vp), C.POINTER(vp),
                                       C.POINTER(SolveOpts), ip, C.c_void_p, ip, vp]),
        "biot_sizes": (C.c_int, [vp, i64p, i64p, i64p]),
        "biot_time_tables": (C.c_int, [C.c_int, dp, dp, dp, dp, dp, dp, dp, ip, dp]),
        "biot_set_permeability": (C.c_int, [vp, dp]),
        "biot_set_log_permeability": (C.c_int, [vp, dp, C.c_double]),
        "biot_apply_slab": (C.c_int, [vp, C.c_double, vp, vp, C.c_int, C.c_int, vp]),
        "biot_precondition": (C.c_int, [vp, C.c_double, vp, vp, C.c_int, C.c_int, vp]),
        "biot_solve_slab": (C.c_int, [vp, C.c_double, vp, vp, C.POINTER(SolveOpts), C.POINTER(Stats), vp]),
        "biot_march": (C.c_int, [vp, C.c_double, C.c_int, C.c_int, C.POINTER(vp), dp, vp, vp, vp,
                                 C.POINTER(SolveOpts), ip, C.POINTER(Stats), vp]),
        "biot_march_resume": (C.c_int, [vp, C.c_double, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(vp), dp, vp, vp, vp,
                                        C.POINTER(SolveOpts), ip, C.POINTER(Stats), vp]),
        "biot_adjoint_grad": (C.c_int, [vp, C.c_double, C.c_int, C.c_int, C.POINTER(vp), dp, vp, vp,
                                        C.POINTER(SolveOpts), C.c_int, dp, vp, vp]),
        "biot_goal_mean_pressure": (C.c_int, [vp, dp, dp, vp, vp]),
        "biot_dwr_time_estimate": (C.c_int, [vp, vp, C.c_double, C.c_int, C.c_int, C.POINTER(vp), dp, vp, vp,
                                             C.POINTER(SolveOpts), dp, dp, dp, vp]),
        "biot_solve_batch": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(Opts), C.POINTER(SolveOpts), C.c_int, ip,
                                       C.c_void_p]),
        "biot_load_preset": (C.c_int, [vp, C.c_int, C.c_double, vp, vp]),
        "biot_apply_part": (C.c_int, [vp, C.c_int, C.c_double, vp, vp, C.c_int, vp]),
        "biot_schur_apply_noalloc": (C.c_int, [vp, C.c_double, vp, vp, vp]),
        "biot_profile": (C.c_int, [vp, C.c_int]),
        "biot_kernel_stats": (C.c_int, [vp, C.c_int, i64p, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
        "biot_counters": (C.c_int, [vp, i64p, i64p, C.POINTER(C.c_double)]),
        "biot_fma_peak": (C.c_int, [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), vp]),
        "biot_schur_bounds": (C.c_int, [vp, C.c_double, dp, ip, vp]),
        "biot_tune_get": (C.c_int, [C.c_char_p]),
        "biot_tune_put": (C.c_int, [C.c_char_p, C.c_int]),
        "biot_tune_cache_path": (C.c_int, [C.c_char_p, C.c_int]),
        "biot_last_error": (C.c_char_p, [vp]),
        "biot_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class BiotError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (ERR_NAMES.get(code, code), msg))
        self.code = code


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t, dtype=None, numel=None, name="tensor"):
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch tensor" % name)
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if numel is not None and t.numel() != numel:
        raise ValueError("%s must have %d elements, got %d" % (name, numel, t.numel()))
    return C.c_void_p(t.data_ptr())


def _solve_opts(tol=1e-10, max_iters=2000, mode=FP64, inner_tol=1e-5, transpose=0):
    return SolveOpts(tol, max_iters, mode, inner_tol, transpose)


class Context:
    """One mesh + coefficient set + time order r on the current CUDA device.  With nb > 1
    (biot_setup_batch) the context holds nb instances that differ only in their
    permeability (coeffs["K"]: nb * n_cells values, instance-major) and in their loads;
    its slab vectors are level-major (level k of instance b at (k * nb + b) * n_space)."""

    def __init__(self, dim, n, coeffs: dict, r: int, u_bc, f_bc, lo=None, hi=None, opts: dict | None = None, nb: int = 1):
        lib = load()
        m = Mesh()
        m.dim = dim
        for d in range(3):
            m.n[d] = int(n[d]) if d < dim else 1
            m.lo[d] = float(lo[d]) if (lo is not None and d < dim) else 0.0
            m.hi[d] = float(hi[d]) if (hi is not None and d < dim) else 1.0
        for f in range(6):
            m.u_bc[f] = int(u_bc[f]) if f < 2 * dim else 0
            m.f_bc[f] = int(f_bc[f]) if f < 2 * dim else 0
        self.K = np.ascontiguousarray(np.asarray(coeffs["K"], dtype=np.float64))
        co = Coeffs(coeffs["b"], coeffs["invM"], coeffs["K_dr"], coeffs["lam"], coeffs["mu"], coeffs["eta"],
                    self.K.ctypes.data_as(C.POINTER(C.c_double)))
        o = Opts(0, 0, 0, 0, -1.0, 0, 0, 0)
        if opts:
            for k, v in opts.items():
                setattr(o, k, v)
        h = C.c_void_p()
        if nb == 1:
            rc = lib.biot_setup(C.byref(m), C.byref(co), int(r), C.byref(o), C.byref(h))
        else:
            rc = lib.biot_setup_batch(C.byref(m), C.byref(co), int(r), C.byref(o), int(nb), C.byref(h))
        if rc != OK:
            raise BiotError(rc, lib.biot_last_error(None).decode())
        self.h = h
        self.lib = lib
        self.nb = int(nb)
        self.dim, self.r, self.nt = dim, r, r + 1
        ns, nsl, nc = C.c_int64(), C.c_int64(), C.c_int64()
        lib.biot_sizes(h, C.byref(ns), C.byref(nsl), C.byref(nc))
        # per-instance sizes; a batched slab vector holds nb of them (n_slab_all)
        self.n_space, self.n_slab, self.n_cells = ns.value, nsl.value, nc.value
        self.n_slab_all = self.n_slab * self.nb

    def _check(self, rc, allow=()):
        if rc != OK and rc not in allow:
            raise BiotError(rc, self.lib.biot_last_error(self.h).decode())
        return rc

    def destroy(self):
        if getattr(self, "h", None):
            self.lib.biot_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    # --- entry points (names follow include/biot.h) ---
    def set_permeability(self, K):
        self.K = np.ascontiguousarray(np.asarray(K, dtype=np.float64))
        assert self.K.size == self.n_cells
        return self._check(self.lib.biot_set_permeability(self.h, self.K.ctypes.data_as(C.POINTER(C.c_double))))

    def set_log_permeability(self, g, K0):
        """K = K0 exp(g) per cell, formed by the library (biot_set_log_permeability)."""
        g = np.ascontiguousarray(np.asarray(g, dtype=np.float64))
        assert g.size == self.n_cells * self.nb
        rc = self._check(self.lib.biot_set_log_permeability(self.h, g.ctypes.data_as(C.POINTER(C.c_double)), float(K0)))
        return rc

    def apply_slab(self, tau, x, y, transpose=False):
        import torch
        prec = FP64 if x.dtype == torch.float64 else FP32
        dt = torch.float64 if prec == FP64 else torch.float32
        return self._check(self.lib.biot_apply_slab(self.h, float(tau), _ptr(x, dt, self.n_slab_all, "x"),
                                                    _ptr(y, dt, self.n_slab_all, "y"), prec, int(transpose), _stream()))

    def precondition(self, tau, r, z, transpose=False):
        import torch
        prec = FP64 if r.dtype == torch.float64 else FP32
        dt = torch.float64 if prec == FP64 else torch.float32
        return self._check(self.lib.biot_precondition(self.h, float(tau), _ptr(r, dt, self.n_slab_all, "r"),
                                                      _ptr(z, dt, self.n_slab_all, "z"), prec, int(transpose), _stream()))

    def solve_slab(self, tau, rhs, x, tol=1e-10, max_iters=2000, mode=FP64, inner_tol=1e-5, transpose=False,
                   allow_noconv=False):
        import torch
        st = Stats()
        o = _solve_opts(tol, max_iters, mode, inner_tol, int(transpose))
        rc = self.lib.biot_solve_slab(self.h, float(tau), _ptr(rhs, torch.float64, self.n_slab, "rhs"),
                                      _ptr(x, torch.float64, self.n_slab, "x"), C.byref(o), C.byref(st), _stream())
        self._check(rc, allow=(ENOCONV,) if allow_noconv else ())
        return st.as_dict()

    def _loads(self, f_terms, tcoef):
        nterms = len(f_terms)
        arr = (C.c_void_p * max(1, nterms))()
        keep = []
        for i, f in enumerate(f_terms):
            if isinstance(f, np.ndarray):
                f = np.ascontiguousarray(f, dtype=np.float64)
                assert f.size == self.n_space
                keep.append(f)
                arr[i] = f.ctypes.data
            else:
                arr[i] = _ptr(f, None, self.n_space, "f_term").value
                keep.append(f)
        tc = np.ascontiguousarray(np.asarray(tcoef, dtype=np.float64).reshape(-1)) if nterms else np.zeros(4)
        assert tc.size == 4 * max(1, nterms) or nterms == 0
        return nterms, arr, tc, keep

    def march(self, T, slabs, f_terms, tcoef, U0, U_end, X_all=None, tol=1e-10, max_iters=2000, mode=FP64,
              inner_tol=1e-5, allow_noconv=False):
        """U0 / U_end may be torch CUDA tensors or (pinned) CPU tensors / numpy arrays."""
        nterms, arr, tc, keep = self._loads(f_terms, tcoef)
        o = _solve_opts(tol, max_iters, mode, inner_tol, 0)
        st = Stats()
        its = (C.c_int * slabs)()

        def anyptr(t, name):
            if t is None:
                return None
            if isinstance(t, np.ndarray):
                assert t.dtype == np.float64 and t.flags.c_contiguous and t.size == self.n_space, name
                return C.c_void_p(t.ctypes.data)
            return _ptr(t, None, self.n_space, name)
        rc = self.lib.biot_march(self.h, float(T), int(slabs), nterms, arr, tc.ctypes.data_as(C.POINTER(C.c_double)),
                                 anyptr(U0, "U0"), anyptr(U_end, "U_end"),
                                 _ptr(X_all, None, None, "X_all"), C.byref(o), its, C.byref(st), _stream())
        self._check(rc, allow=(ENOCONV,) if allow_noconv else ())
        d = st.as_dict()
        d["iters_per_slab"] = list(its)
        return d

    def march_resume(self, T, slabs, first, count, f_terms, tcoef, U_first, U_end, X_all=None, tol=1e-10, max_iters=2000,
                     mode=FP64, inner_tol=1e-5, allow_noconv=False):
        """Slabs first .. first+count-1 of the partition of (0, T] into `slabs` slabs, from
        U_first = U(t_first^-) (biot_march_resume)."""
        nterms, arr, tc, keep = self._loads(f_terms, tcoef)
        o = _solve_opts(tol, max_iters, mode, inner_tol, 0)
        st = Stats()
        its = (C.c_int * count)()

        def anyptr(t, name):
            if isinstance(t, np.ndarray):
                assert t.dtype == np.float64 and t.flags.c_contiguous and t.size == self.n_space, name
                return C.c_void_p(t.ctypes.data)
            return _ptr(t, None, self.n_space, name)
        rc = self.lib.biot_march_resume(self.h, float(T), int(slabs), int(first), int(count), nterms, arr,
                                        tc.ctypes.data_as(C.POINTER(C.c_double)), anyptr(U_first, "U_first"),
                                        anyptr(U_end, "U_end"), _ptr(X_all, None, None, "X_all"), C.byref(o), its,
                                        C.byref(st), _stream())
        self._check(rc, allow=(ENOCONV,) if allow_noconv else ())
        d = st.as_dict()
        d["iters_per_slab"] = list(its)
        return d

    def march_batch(self, T, slabs, f_terms, tcoef, U0, U_end, tol=1e-10, max_iters=2000, inner_tol=1e-5):
        """Batched march (biot_march_batch, BIOT_MIXED).  f_terms: one list of load terms per
        instance (same count for all; torch CUDA tensors or numpy arrays of n_space);
        U0: None or one state per instance; U_end: one output per instance (torch CUDA tensor
        or float64 numpy array).  Returns (rc, status list, stats dicts)."""
        nb = self.nb
        assert len(f_terms) == nb and len(U_end) == nb
        nterms = len(f_terms[0])
        flat = [f for terms in f_terms for f in terms]
        assert len(flat) == nb * nterms
        arr = (C.c_void_p * max(1, nb * nterms))()
        keep = []

        def anyptr(t, name):
            if t is None:
                return None
            if isinstance(t, np.ndarray):
                assert t.dtype == np.float64 and t.flags.c_contiguous and t.size == self.n_space, name
                keep.append(t)
                return t.ctypes.data
            keep.append(t)
            return _ptr(t, None, self.n_space, name).value
        for i, f in enumerate(flat):
            if isinstance(f, np.ndarray):
                f = np.ascontiguousarray(f, dtype=np.float64)
            arr[i] = anyptr(f, "f_term")
        tc = np.ascontiguousarray(np.asarray(tcoef, dtype=np.float64).reshape(-1)) if nterms else np.zeros(4)
        u0 = (C.c_void_p * nb)(*[anyptr(u, "U0") for u in U0]) if U0 is not None else None
        ue = (C.c_void_p * nb)(*[anyptr(u, "U_end") for u in U_end])
        o = _solve_opts(tol, max_iters, MIXED, inner_tol, 0)
        its = (C.c_int * nb)()
        stats = (Stats * nb)()
        status = (C.c_int * nb)()
        rc = self.lib.biot_march_batch(self.h, float(T), int(slabs), nterms, arr, tc.ctypes.data_as(C.POINTER(C.c_double)),
                                       u0, ue, C.byref(o), its, C.cast(stats, C.c_void_p), status, _stream())
        return rc, list(status), [s.as_dict() for s in stats]

    def adjoint_grad(self, T, slabs, f_terms, tcoef, U0, j_goal, dJ, tol=1e-10, max_iters=2000, mode=FP64,
                     inner_tol=1e-5, recompute=True):
        import torch
        nterms, arr, tc, keep = self._loads(f_terms, tcoef)
        o = _solve_opts(tol, max_iters, mode, inner_tol, 0)
        J = C.c_double()
        rc = self.lib.biot_adjoint_grad(self.h, float(T), int(slabs), nterms, arr,
                                        tc.ctypes.data_as(C.POINTER(C.c_double)),
                                        _ptr(U0, torch.float64, self.n_space, "U0"),
                                        _ptr(j_goal, torch.float64, self.n_space, "j_goal"), C.byref(o),
                                        int(bool(recompute)), C.byref(J), _ptr(dJ, torch.float64, self.n_cells, "dJ"),
                                        _stream())
        self._check(rc)
        return J.value

    def dwr_time_estimate(self, ctx_r1, T, slabs, f_terms, tcoef, U0, j_goal, tol=1e-10, max_iters=2000, mode=FP64,
                          inner_tol=1e-5):
        """Dual-weighted residual estimate of the dG(r) time error of J = j^T U(T^-) against
        dG(r+1) (biot_dwr_time_estimate).  Returns (eta, per-slab indicators, J(U_r))."""
        import torch
        nterms, arr, tc, keep = self._loads(f_terms, tcoef)
        o = _solve_opts(tol, max_iters, mode, inner_tol, 0)
        eta_s = (C.c_double * slabs)()
        eta, J = C.c_double(), C.c_double()
        rc = self.lib.biot_dwr_time_estimate(self.h, ctx_r1.h, float(T), int(slabs), nterms, arr,
                                             tc.ctypes.data_as(C.POINTER(C.c_double)),
                                             _ptr(U0, torch.float64, self.n_space, "U0"),
                                             _ptr(j_goal, torch.float64, self.n_space, "j_goal"), C.byref(o), eta_s,
                                             C.byref(eta), C.byref(J), _stream())
        self._check(rc)
        return eta.value, list(eta_s), J.value

    def goal_mean_pressure(self, lo, hi, j):
        import torch
        lo = (C.c_double * 3)(*[float(v) for v in lo] + [0.0] * (3 - len(lo)))
        hi = (C.c_double * 3)(*[float(v) for v in hi] + [0.0] * (3 - len(hi)))
        return self._check(self.lib.biot_goal_mean_pressure(self.h, lo, hi, _ptr(j, torch.float64, self.n_space, "j"),
                                                            _stream()))

    def apply_part(self, part, tau, x, y):
        import torch
        prec = FP64 if x.dtype == torch.float64 else FP32
        dt = torch.float64 if prec == FP64 else torch.float32
        return self._check(self.lib.biot_apply_part(self.h, int(part), float(tau), _ptr(x, dt, self.n_space, "in"),
                                                    _ptr(y, dt, self.n_space, "out"), prec, _stream()))

    def schur_apply_noalloc(self, tau, x, y):
        """Allocation-free flux-pressure Schur apply (FP64 spatial vectors)."""
        import torch
        return self._check(self.lib.biot_schur_apply_noalloc(self.h, float(tau), _ptr(x, torch.float64, self.n_space, "in"),
                                                             _ptr(y, torch.float64, self.n_space, "out"), _stream()))

    def schur_bounds(self, tau):
        """(smallest Ritz value, largest Ritz value, Chebyshev interval lo, hi, degree) of the
        Jacobi-scaled lumped Schur complement for this tau (biot_schur_bounds)."""
        b = (C.c_double * 4)()
        deg = C.c_int()
        self._check(self.lib.biot_schur_bounds(self.h, float(tau), b, C.byref(deg), _stream()))
        return tuple(b) + (deg.value,)

    def profile(self, enable):
        return self._check(self.lib.biot_profile(self.h, int(bool(enable))))

    def counters(self):
        """(kernel launches so far, recorded operator launches, their device ms)."""
        a, b, ms = C.c_int64(), C.c_int64(), C.c_double()
        self._check(self.lib.biot_counters(self.h, C.byref(a), C.byref(b), C.byref(ms)))
        return a.value, b.value, ms.value

    def kernel_stats(self, kind):
        """(launches, device ms, work units) of the recorded launches of one kernel kind."""
        n, ms, u = C.c_int64(), C.c_double(), C.c_double()
        self._check(self.lib.biot_kernel_stats(self.h, int(kind), C.byref(n), C.byref(ms), C.byref(u)))
        return n.value, ms.value, u.value

    def load_preset(self, kind, value, f):
        import torch
        return self._check(self.lib.biot_load_preset(self.h, int(kind), float(value),
                                                     _ptr(f, torch.float64, self.n_space, "f"), _stream()))


def _goal_function_class():
    import torch

    class GoalOfLogK(torch.autograd.Function):
        """J(g) = j^T U(T^-) as a differentiable function of the cellwise log-permeability g
        (K = K0 exp(g)).  forward runs biot_adjoint_grad, which returns J and dJ/dg together
        (the dual problem marched backwards with checkpoint recomputation); backward scales
        that gradient by the incoming one.  No arithmetic of the method runs in Python."""

        @staticmethod
        def forward(fctx, g, context, K0, T, slabs, f_terms, tcoef, U0, j_goal, tol, mode):
            gh = np.ascontiguousarray(g.detach().to("cpu", torch.float64).numpy())
            context.set_log_permeability(gh, K0)
            dJ = torch.zeros(context.n_cells, dtype=torch.float64, device=j_goal.device)
            J = context.adjoint_grad(T, slabs, f_terms, tcoef, U0, j_goal, dJ, tol=tol, mode=mode)
            fctx.save_for_backward(dJ)
            return torch.tensor(J, dtype=torch.float64, device=g.device)

        @staticmethod
        def backward(fctx, gout):
            (dJ,) = fctx.saved_tensors
            return (gout * dJ).to(gout.device), None, None, None, None, None, None, None, None, None, None

    return GoalOfLogK


_GOAL = None


def goal_of_logk(context, g, K0, T, slabs, f_terms, tcoef, U0, j_goal, tol=1e-10, mode=FP64):
    """Differentiable goal functional J(g) (torch scalar); g: float64 tensor of n_cells."""
    global _GOAL
    if _GOAL is None:
        _GOAL = _goal_function_class()
    return _GOAL.apply(g, context, K0, T, slabs, f_terms, tcoef, U0, j_goal, tol, mode)


def fma_peak(prec=FP32):
    """Measured CUDA-core FMA throughput of the current device (biot_fma_peak):
    (TFLOP/s, ms of the timed launch)."""
    lib = load()
    tf, ms = C.c_double(), C.c_double()
    rc = lib.biot_fma_peak(int(prec), C.byref(tf), C.byref(ms), _stream())
    if rc != OK:
        raise BiotError(rc, "biot_fma_peak failed")
    return tf.value, ms.value


def tune_get(key):
    """Stored launch-shape choice for `key` (biot_tune_get), or -1."""
    return int(load().biot_tune_get(key.encode()))


def tune_put(key, value):
    """Store a launch-shape choice (biot_tune_put); also written to the cache file."""
    rc = load().biot_tune_put(key.encode(), int(value))
    if rc != OK:
        raise BiotError(rc, "biot_tune_put: invalid key %r" % key)


def tune_cache_path():
    """Path of the tuning cache file this process reads and writes (biot_tune_cache_path)."""
    buf = C.create_string_buffer(4096)
    rc = load().biot_tune_cache_path(buf, len(buf))
    if rc != OK:
        raise BiotError(rc, "biot_tune_cache_path failed")
    return buf.value.decode()


def time_tables(r):
    """Host time tables of dG(r) (biot_time_tables): dict of numpy arrays."""
    lib = load()
    nt = r + 1
    out = {k: np.zeros(nt) for k in ("nodes", "w", "phi0", "lam")}
    out.update({k: np.zeros((nt, nt)) for k in ("D", "V", "W")})
    pair, beta = C.c_int(), C.c_double()
    dptr = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))  # noqa: E731
    rc = lib.biot_time_tables(int(r), dptr(out["nodes"]), dptr(out["w"]), dptr(out["phi0"]), dptr(out["D"]), dptr(out["V"]),
                              dptr(out["W"]), dptr(out["lam"]), C.byref(pair), C.byref(beta))
    if rc != OK:
        raise BiotError(rc, "biot_time_tables")
    out["pair"], out["pair_beta"] = pair.value, beta.value
    return out


def make_mesh(dim, n, u_bc, f_bc, lo=None, hi=None):
    m = Mesh()
    m.dim = dim
    for d in range(3):
        m.n[d] = int(n[d]) if d < dim else 1
        m.lo[d] = float(lo[d]) if (lo is not None and d < dim) else 0.0
        m.hi[d] = float(hi[d]) if (hi is not None and d < dim) else 1.0
    for f in range(6):
        m.u_bc[f] = int(u_bc[f]) if f < 2 * dim else 0
        m.f_bc[f] = int(f_bc[f]) if f < 2 * dim else 0
    return m


def solve_batch(instances, workers=0, tol=1e-10, mode=MIXED, inner_tol=1e-5, max_iters=2000, opts=None):
    """Batched marches (biot_solve_batch).  Each instance is a dict with dim, n, coeffs
    (b, invM, K_dr, lam, mu, eta, K), r, T, slabs, u_bc, f_bc, load_kind, load_value and
    U_end (a float64 numpy array of n_space that receives the end state).  `workers`:
    at most this many instances per batched context (0: the library default).
    Returns (rc, per-instance status list, per-instance stats dicts)."""
    lib = load()
    cnt = len(instances)
    items = (BatchItem * cnt)()
    keep = []
    for i, ins in enumerate(instances):
        it = items[i]
        it.mesh = make_mesh(ins["dim"], ins["n"], ins["u_bc"], ins["f_bc"])
        K = np.ascontiguousarray(np.asarray(ins["coeffs"]["K"], dtype=np.float64))
        keep.append(K)
        co = ins["coeffs"]
        it.coeffs = Coeffs(co["b"], co["invM"], co["K_dr"], co["lam"], co["mu"], co["eta"],
                           K.ctypes.data_as(C.POINTER(C.c_double)))
        it.r, it.T, it.slabs = int(ins["r"]), float(ins["T"]), int(ins["slabs"])
        it.load_kind, it.load_value, it.nterms = int(ins.get("load_kind", 0)), float(ins.get("load_value", 1.0)), 0
        it.f_terms = None
        it.tcoef = None
        it.U0 = None
        out = ins.get("U_end")
        it.U_end = out.ctypes.data if out is not None else None
    o = Opts(0, 0, 0, 0, -1.0, 0, 0, 0)
    if opts:
        for k, v in opts.items():
            setattr(o, k, v)
    so = SolveOpts(tol, max_iters, mode, inner_tol, 0)
    status = (C.c_int * cnt)()
    stats = (Stats * cnt)()
    rc = lib.biot_solve_batch(C.cast(items, C.c_void_p), cnt, C.byref(o), C.byref(so), int(workers), status,
                              C.cast(stats, C.c_void_p))
    return rc, list(status), [s.as_dict() for s in stats]
