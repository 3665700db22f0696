"""ctypes binding of libelrt.so (argument marshalling only)."""

from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libelrt.so")
HEADER = os.path.join(HERE, "..", "include", "elrt.h")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2308_02467_gb300.build`")
_lib = C.CDLL(LIB_PATH)

ANG_FV0, ANG_DO = 0, 1
LOCAL_FP64, LOCAL_FP32_IR, LOCAL_TF32_IR = 0, 1, 2
F32, F64 = 0, 1
KRYLOV_F32, KRYLOV_F16 = 0, 1
PRECOND_NONE, PRECOND_SWEEP = 0, 1
LU_PRODUCTS_AUTO, LU_PRODUCTS_TF32 = 0, 1
STATUS = {0: "ok", 1: "EINVAL", 2: "ENOMEM", 3: "ESINGULAR", 4: "ENOCONV", 5: "ETIMEOUT", 6: "ECUDA", 7: "ENOTRAINED"}


class Disc(C.Structure):
    _fields_ = [("p", C.c_int32), ("n_angles", C.c_int32), ("angular", C.c_int32), ("hg_g", C.c_double)]


class LocalStats(C.Structure):
    _fields_ = [("refine_steps", C.c_int32), ("n_flagged", C.c_int32), ("max_rel_residual", C.c_double)]


class LocalExtras(C.Structure):
    _fields_ = [("source", C.c_void_p), ("f2o", C.c_void_p), ("f2m", C.c_void_p), ("f2u", C.c_void_p),
                ("in2rad", C.c_void_p)]


class TuneReport(C.Structure):
    _fields_ = [("local_chunk", C.c_int64), ("lu_pairs", C.c_int32), ("restart", C.c_int32),
                ("n_candidates", C.c_int32), ("local_ms_default", C.c_double), ("local_ms_best", C.c_double),
                ("solve_ms_default", C.c_double), ("solve_ms_best", C.c_double)]


class SolveStats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("restarts", C.c_int32), ("converged", C.c_int32),
                ("rel_residual", C.c_double)]


class NetDesc(C.Structure):
    _fields_ = [("p", C.c_int32), ("n_angles", C.c_int32), ("n_hidden", C.c_int32), ("width", C.c_int32),
                ("activation", C.c_int32), ("seed", C.c_uint64), ("features", C.c_int32)]


class TrainOpts(C.Structure):
    _fields_ = [("epochs", C.c_int32), ("batch", C.c_int32), ("lr", C.c_float), ("beta1", C.c_float),
                ("beta2", C.c_float), ("eps", C.c_float), ("seed", C.c_uint64)]


class Field(C.Structure):
    _fields_ = [("nx", C.c_int32), ("nz", C.c_int32), ("h", C.c_double), ("kappa", C.c_void_p),
                ("omega", C.c_void_p), ("inflow", C.c_void_p)]


class SolveOpts(C.Structure):
    _fields_ = [("mode", C.c_int32), ("refine_steps", C.c_int32), ("rtol", C.c_double), ("max_iter", C.c_int32),
                ("restart", C.c_int32), ("net", C.c_void_p), ("learned_tol", C.c_double)]


class FieldStats(C.Structure):
    _fields_ = [("local", LocalStats), ("glob", SolveStats), ("n_fallback", C.c_int64), ("local_ms", C.c_double),
                ("global_ms", C.c_double)]


class ElrtError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_vp, _i32, _i64, _d = C.c_void_p, C.c_int32, C.c_int64, C.c_double
_P = C.POINTER
_sig = {
    "elrt_n_nodes": (_i64, [_P(Disc)]),
    "elrt_n_local": (_i64, [_P(Disc)]),
    "elrt_n_skel": (_i64, [_P(Disc)]),
    "elrt_n_inflow": (_i64, [_P(Disc), _i32, _i32]),
    "elrt_lgl": (_i32, [_i32, _vp, _vp]),
    "elrt_phase_matrix": (_i32, [_P(Disc), _vp]),
    "elrt_node_coords": (_i32, [_P(Disc), _i32, _i32, _d, _vp, _vp]),
    "elrt_create": (_i32, [_P(_vp), _P(Disc), _vp]),
    "elrt_destroy": (_i32, [_vp]),
    "elrt_set_stream": (_i32, [_vp, _vp]),
    "elrt_set_krylov_op": (_i32, [_vp, _i32]),
    "elrt_set_graphs": (_i32, [_vp, _i32]),
    "elrt_set_precond": (_i32, [_vp, _i32]),
    "elrt_set_lu_products": (_i32, [_vp, _i32]),
    "elrt_apply_precond": (_i32, [_vp, _i32, _i32, _vp, _i32, _vp, _vp]),
    "elrt_autotune": (_i32, [_vp, _P(Field), _i32, _i32, _d, _P(TuneReport)]),
    "elrt_get_tuning": (_i32, [_vp, _P(_i64), _P(_i32), _P(_i32), _P(_i32)]),
    "elrt_set_tuning": (_i32, [_vp, _i64, _i32, _i32]),
    "elrt_status_str": (C.c_char_p, [_i32]),
    "elrt_last_error": (C.c_char_p, [_vp]),
    "elrt_assemble": (_i32, [_vp, _i64, _d, _vp, _vp, _vp, _vp, _vp]),
    "elrt_build_local": (_i32, [_vp, _i64, _d, _vp, _vp, _vp, _i32, _i32, _i32, _vp, _vp, _vp, _P(LocalStats)]),
    "elrt_build_local_ex": (_i32, [_vp, _i64, _d, _vp, _vp, _vp, _i32, _i32, _i32, _vp, _vp, _P(LocalExtras), _vp,
                                   _P(LocalStats)]),
    "elrt_solve_global_source": (_i32, [_vp, _i32, _i32, _vp, _i32, _vp, _vp, _d, _i32, _i32, _i32, _vp,
                                        _P(SolveStats)]),
    "elrt_recover_mean_source": (_i32, [_vp, _i32, _i32, _vp, _i32, _vp, _vp, _vp, _vp]),
    "elrt_recover_radiance": (_i32, [_vp, _i32, _i32, _vp, _i32, _vp, _vp, _vp, _vp]),
    "elrt_global_apply": (_i32, [_vp, _i32, _i32, _vp, _i32, _vp, _vp]),
    "elrt_solve_global": (_i32, [_vp, _i32, _i32, _vp, _i32, _vp, _d, _i32, _i32, _i32, _vp, _P(SolveStats)]),
    "elrt_recover_mean": (_i32, [_vp, _i32, _i32, _vp, _i32, _vp, _vp, _vp]),
    "elrt_profile_enable": (_i32, [_vp, _i32]),
    "elrt_profile_reset": (_i32, [_vp]),
    "elrt_profile_get": (_i32, [_vp, C.c_char_p, _P(_d), _P(_i64)]),
    "elrt_profile_work": (_i32, [_vp, C.c_char_p, _P(_d), _P(_d)]),
    "elrt_launch_count": (_i64, [_vp]),
    "elrt_build_local_static": (_i32, [_P(Disc), _vp, _i64, _d, _vp, _vp, _vp, _i32, _i32, _i32, _vp, _vp]),
    "elrt_solve_field": (_i32, [_vp, _P(Field), _P(SolveOpts), _vp, _vp, _P(FieldStats)]),
    "elrt_solve_batch": (_i32, [_P(_vp), _i32, _P(Field), _P(_i32), _i32, _P(SolveOpts), C.c_size_t, _i32, _P(_vp),
                                 _P(FieldStats)]),
    "elrt_net_create": (_i32, [_P(_vp), _P(NetDesc), _vp]),
    "elrt_net_destroy": (_i32, [_vp]),
    "elrt_net_set_stream": (_i32, [_vp, _vp]),
    "elrt_net_last_error": (C.c_char_p, [_vp]),
    "elrt_net_sizes": (_i32, [_vp, _P(_i64), _P(_i64), _P(_i64), _P(_i32), _P(_i64)]),
    "elrt_net_params": (_i32, [_vp, _i32, _i32, _i32, _vp]),
    "elrt_net_save": (_i32, [_vp, C.c_char_p]),
    "elrt_net_load": (_i32, [_P(_vp), C.c_char_p, _vp]),
    "elrt_net_file_info": (_i32, [C.c_char_p, _P(NetDesc), _P(_i32), _P(_i64), _P(_i64)]),
    "elrt_net_forward": (_i32, [_vp, _i64, _vp, _vp]),
    "elrt_net_train_step": (_i32, [_vp, _i64, _vp, _vp, C.c_float, _P(C.c_float)]),
    "elrt_net_fit": (_i32, [_vp, _i64, _vp, _vp, _vp, _vp, _vp, _P(TrainOpts), _vp]),
    "elrt_net_infer": (_i32, [_vp, _i64, _d, _vp, _vp, _vp, _vp, _vp]),
    "elrt_build_local_learned": (_i32, [_vp, _vp, _i64, _d, _vp, _vp, _vp, _d, _vp, _vp, _vp, _P(_i64)]),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def exported_symbols() -> list[str]:
    """Names of the entry points declared in include/elrt.h (each must resolve in the library)."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(elrt_[a-z0-9_]+)\s*\(", text)))


def _check(status, ctx=None):
    if status != 0:
        msg = _lib.elrt_last_error(ctx)
        raise ElrtError(status, msg.decode() if msg else "")


def _disc(p, n_angles, hg_g=0.0, angular=ANG_FV0) -> Disc:
    return Disc(int(p), int(n_angles), int(angular), float(hg_g))


# ----------------------------------------------------------------------------- host helpers
def elrt_n_nodes(p, n_angles):
    return _lib.elrt_n_nodes(C.byref(_disc(p, n_angles)))


def elrt_n_local(p, n_angles):
    return _lib.elrt_n_local(C.byref(_disc(p, n_angles)))


def elrt_n_skel(p, n_angles):
    return _lib.elrt_n_skel(C.byref(_disc(p, n_angles)))


def elrt_n_inflow(p, n_angles, nx, nz):
    return _lib.elrt_n_inflow(C.byref(_disc(p, n_angles)), nx, nz)


def elrt_lgl(p):
    xi = np.zeros(p + 1)
    w = np.zeros(p + 1)
    _check(_lib.elrt_lgl(p, xi.ctypes.data, w.ctypes.data))
    return xi, w


def elrt_phase_matrix(n_angles, hg_g, angular=ANG_FV0):
    W = np.zeros((n_angles, n_angles))
    _check(_lib.elrt_phase_matrix(C.byref(_disc(1, n_angles, hg_g, angular)), W.ctypes.data))
    return W


def elrt_node_coords(p, n_angles, nx, nz, h):
    nm = (p + 1) ** 2
    x = np.zeros((nx * nz, nm))
    z = np.zeros((nx * nz, nm))
    _check(_lib.elrt_node_coords(C.byref(_disc(p, n_angles)), nx, nz, h, x.ctypes.data, z.ctypes.data))
    return x, z


# ----------------------------------------------------------------------------- device calls
def elrt_build_local_static(p, n_angles, hg_g, angular, kappa, omega, h, in2out, in2sol, mode=LOCAL_FP32_IR,
                            refine_steps=2, h_elem=None):
    """The allocation-free local build (no context; scratch in a fixed device array of the library).
    Returns the status code (0 = ok) instead of raising, so callers can inspect rejections."""
    import torch
    E = omega.numel()
    nm, nin = (p + 1) ** 2, 2 * (p + 1) * n_angles
    d = _disc(p, n_angles, hg_g, angular)
    return _lib.elrt_build_local_static(
        C.byref(d), C.c_void_p(torch.cuda.current_stream().cuda_stream), E, float(h),
        _ptr(h_elem, torch.float64, E, "h_elem"), _ptr(kappa, torch.float64, E * nm, "kappa"),
        _ptr(omega, torch.float64, E, "omega"), int(mode), int(refine_steps), _dt(in2out),
        _ptr(in2out, None, E * nin * nin, "in2out"), _ptr(in2sol, None, E * nm * nin, "in2sol"))



def _ptr(t, dtype=None, n=None, name="tensor"):
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} must have {n} elements, got {t.numel()}")
    return t.data_ptr()


def _dt(t):
    import torch
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.float64:
        return F64
    raise ValueError("operators must be float32 or float64")


class Context:
    """An elrt_ctx for one discretisation; calls run on the current torch CUDA stream."""

    def __init__(self, p, n_angles, hg_g=0.0, angular=ANG_FV0):
        import torch
        self.disc = _disc(p, n_angles, hg_g, angular)
        self.p, self.n_angles, self.hg_g, self.angular = p, n_angles, hg_g, angular
        self.nm = (p + 1) ** 2
        self.nu = self.nm * n_angles
        self.nin = 2 * (p + 1) * n_angles
        h = C.c_void_p()
        _check(_lib.elrt_create(C.byref(h), C.byref(self.disc), C.c_void_p(torch.cuda.current_stream().cuda_stream)))
        self._h = h

    def _sync_stream(self):
        import torch
        _lib.elrt_set_stream(self._h, C.c_void_p(torch.cuda.current_stream().cuda_stream))

    def close(self):
        if getattr(self, "_h", None):
            _lib.elrt_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- measurement
    def elrt_profile_enable(self, on=True):
        _check(_lib.elrt_profile_enable(self._h, int(bool(on))), self._h)

    def elrt_profile_reset(self):
        _check(_lib.elrt_profile_reset(self._h), self._h)

    def elrt_profile_get(self, kernel):
        ms, n = C.c_double(), C.c_int64()
        _check(_lib.elrt_profile_get(self._h, kernel.encode(), C.byref(ms), C.byref(n)), self._h)
        return ms.value, n.value

    def elrt_profile_work(self, kernel):
        """(algorithmic bytes, useful flops) of the timed launches of one kernel group."""
        b, f = C.c_double(), C.c_double()
        _check(_lib.elrt_profile_work(self._h, kernel.encode(), C.byref(b), C.byref(f)), self._h)
        return b.value, f.value

    def elrt_launch_count(self):
        return _lib.elrt_launch_count(self._h)

    def elrt_autotune(self, nx, nz, h, kappa, omega, inflow, mode=LOCAL_TF32_IR, refine_steps=1, rtol=1e-8):
        """Measures the context's launch parameters on this field and keeps the fastest; returns the
        report as a dict."""
        self._sync_stream()
        f = _field(self, nx, nz, h, kappa, omega, inflow)
        r = TuneReport()
        _check(_lib.elrt_autotune(self._h, C.byref(f), int(mode), int(refine_steps), float(rtol), C.byref(r)), self._h)
        return {k: getattr(r, k) for k, _ in TuneReport._fields_}

    def elrt_get_tuning(self):
        c, p_, r, t = C.c_int64(), C.c_int32(), C.c_int32(), C.c_int32()
        _check(_lib.elrt_get_tuning(self._h, C.byref(c), C.byref(p_), C.byref(r), C.byref(t)), self._h)
        return {"local_chunk": c.value, "lu_pairs": p_.value, "restart": r.value, "tuned": t.value}

    def elrt_set_tuning(self, local_chunk=0, lu_pairs=1, restart=12):
        _check(_lib.elrt_set_tuning(self._h, int(local_chunk), int(lu_pairs), int(restart)), self._h)

    def elrt_set_graphs(self, on=True):
        """CUDA-graph replay of the GMRES restart cycles (default on)."""
        _check(_lib.elrt_set_graphs(self._h, int(bool(on))), self._h)

    def elrt_set_lu_products(self, mode):
        """LU_PRODUCTS_AUTO (default: 3xFP16 trailing updates when the assembled entries allow) or
        LU_PRODUCTS_TF32 (3xTF32 everywhere)."""
        _check(_lib.elrt_set_lu_products(self._h, int(mode)), self._h)

    def elrt_set_precond(self, kind):
        """PRECOND_SWEEP (default) or PRECOND_NONE: preconditioner of the skeleton GMRES (FP32 in2out)."""
        _check(_lib.elrt_set_precond(self._h, int(kind)), self._h)

    def elrt_apply_precond(self, nx, nz, in2out, r, z):
        """z = M r: the sweep preconditioner once (FP32 in2out, FP32 r and z [E][n_out])."""
        import torch
        n = nx * nz * self.nin
        self._sync_stream()
        _check(_lib.elrt_apply_precond(self._h, nx, nz, _ptr(in2out, torch.float32, n * self.nin, "in2out"), F32,
                                       _ptr(r, torch.float32, n, "r"), _ptr(z, torch.float32, n, "z")), self._h)

    def elrt_set_krylov_op(self, op):
        """KRYLOV_F32 (default) or KRYLOV_F16: operator of the Arnoldi-step matvecs (FP32 in2out)."""
        _check(_lib.elrt_set_krylov_op(self._h, int(op)), self._h)

    # ---- local stage
    def elrt_assemble(self, kappa, omega, h, A, rhs, h_elem=None):
        import torch
        E = omega.numel()
        self._sync_stream()
        _check(_lib.elrt_assemble(self._h, E, float(h), _ptr(h_elem, torch.float64, E, "h_elem"),
                                  _ptr(kappa, torch.float64, E * self.nm, "kappa"),
                                  _ptr(omega, torch.float64, E, "omega"),
                                  _ptr(A, torch.float64, E * self.nu * self.nu, "A"),
                                  _ptr(rhs, torch.float64, E * self.nu * self.nin, "rhs")), self._h)

    def elrt_build_local(self, kappa, omega, h, in2out, in2sol, mode=LOCAL_FP64, refine_steps=2,
                         elem_status=None, h_elem=None, stats=True):
        import torch
        E = omega.numel()
        self._sync_stream()
        st = LocalStats()
        dt = _dt(in2out)
        if in2sol.dtype != in2out.dtype:
            raise ValueError("in2out and in2sol must share a dtype")
        _check(_lib.elrt_build_local(
            self._h, E, float(h), _ptr(h_elem, torch.float64, E, "h_elem"),
            _ptr(kappa, torch.float64, E * self.nm, "kappa"), _ptr(omega, torch.float64, E, "omega"),
            int(mode), int(refine_steps), dt, _ptr(in2out, None, E * self.nin * self.nin, "in2out"),
            _ptr(in2sol, None, E * self.nm * self.nin, "in2sol"),
            _ptr(elem_status, torch.int32, E, "elem_status"), C.byref(st) if stats else None), self._h)
        return st if stats else None

    def elrt_build_local_ex(self, kappa, omega, h, in2out, in2sol, mode=LOCAL_FP64, refine_steps=2, source=None,
                            f2o=None, f2m=None, f2u=None, in2rad=None, elem_status=None, h_elem=None, stats=True):
        """elrt_build_local with a volume source (source [E][N][nm] FP64 -> f2o [E][nin], f2m [E][nm],
        f2u [E][nu], FP64) and/or the full radiance operator in2rad [E][nu][nin]."""
        import torch
        E = omega.numel()
        self._sync_stream()
        st = LocalStats()
        dt = _dt(in2out)
        if in2sol.dtype != in2out.dtype or (in2rad is not None and in2rad.dtype != in2out.dtype):
            raise ValueError("in2out, in2sol and in2rad must share a dtype")
        ex = LocalExtras(_ptr(source, torch.float64, E * self.nu, "source"), _ptr(f2o, torch.float64, E * self.nin, "f2o"),
                         _ptr(f2m, torch.float64, E * self.nm, "f2m"), _ptr(f2u, torch.float64, E * self.nu, "f2u"),
                         _ptr(in2rad, None, E * self.nu * self.nin, "in2rad"))
        _check(_lib.elrt_build_local_ex(
            self._h, E, float(h), _ptr(h_elem, torch.float64, E, "h_elem"),
            _ptr(kappa, torch.float64, E * self.nm, "kappa"), _ptr(omega, torch.float64, E, "omega"),
            int(mode), int(refine_steps), dt, _ptr(in2out, None, E * self.nin * self.nin, "in2out"),
            _ptr(in2sol, None, E * self.nm * self.nin, "in2sol"), C.byref(ex),
            _ptr(elem_status, torch.int32, E, "elem_status"), C.byref(st) if stats else None), self._h)
        return st if stats else None

    # ---- global stage
    def elrt_global_apply(self, nx, nz, in2out, x, y):
        import torch
        n = nx * nz * self.nin
        self._sync_stream()
        _check(_lib.elrt_global_apply(self._h, nx, nz, _ptr(in2out, None, n * self.nin, "in2out"), _dt(in2out),
                                      _ptr(x, torch.float64, n, "x"), _ptr(y, torch.float64, n, "y")), self._h)

    def elrt_solve_global(self, nx, nz, in2out, inflow, skeleton, rtol=1e-10, max_iter=5000, restart=12,
                          use_guess=False, raise_on_noconv=True):
        import torch
        n = nx * nz * self.nin
        self._sync_stream()
        st = SolveStats()
        s = _lib.elrt_solve_global(self._h, nx, nz, _ptr(in2out, None, n * self.nin, "in2out"), _dt(in2out),
                                   _ptr(inflow, torch.float64, 2 * (nx + nz) * (self.p + 1) * (self.n_angles // 2),
                                        "inflow"),
                                   float(rtol), int(max_iter), int(restart), int(bool(use_guess)),
                                   _ptr(skeleton, torch.float64, n, "skeleton"), C.byref(st))
        if s == 4 and not raise_on_noconv:
            return st
        _check(s, self._h)
        return st

    def elrt_solve_field(self, nx, nz, h, kappa, omega, inflow, mean, skeleton=None, mode=LOCAL_FP32_IR,
                         refine_steps=1, rtol=1e-8, max_iter=20000, restart=12, net=None, learned_tol=1e-3,
                         raise_on_noconv=True):
        import torch
        E = nx * nz
        self._sync_stream()
        f = _field(self, nx, nz, h, kappa, omega, inflow)
        o = _opts(mode, refine_steps, rtol, max_iter, restart, net, learned_tol)
        st = FieldStats()
        s = _lib.elrt_solve_field(self._h, C.byref(f), C.byref(o), _ptr(mean, torch.float64, E * self.nm, "mean"),
                                  _ptr(skeleton, torch.float64, E * self.nin, "skeleton"), C.byref(st))
        if not (s == 4 and not raise_on_noconv):
            _check(s, self._h)
        return st

    def elrt_solve_global_source(self, nx, nz, in2out, inflow, f2o, skeleton, rtol=1e-10, max_iter=5000, restart=12,
                                 use_guess=False, raise_on_noconv=True):
        import torch
        n = nx * nz * self.nin
        self._sync_stream()
        st = SolveStats()
        s = _lib.elrt_solve_global_source(self._h, nx, nz, _ptr(in2out, None, n * self.nin, "in2out"), _dt(in2out),
                                          _ptr(inflow, torch.float64, 2 * (nx + nz) * (self.p + 1) * (self.n_angles // 2),
                                               "inflow"),
                                          _ptr(f2o, torch.float64, n, "f2o"), float(rtol), int(max_iter), int(restart),
                                          int(bool(use_guess)), _ptr(skeleton, torch.float64, n, "skeleton"),
                                          C.byref(st))
        if s == 4 and not raise_on_noconv:
            return st
        _check(s, self._h)
        return st

    def elrt_recover_mean_source(self, nx, nz, in2sol, f2m, skeleton, inflow, mean):
        import torch
        E = nx * nz
        self._sync_stream()
        _check(_lib.elrt_recover_mean_source(self._h, nx, nz, _ptr(in2sol, None, E * self.nm * self.nin, "in2sol"),
                                             _dt(in2sol), _ptr(f2m, torch.float64, E * self.nm, "f2m"),
                                             _ptr(skeleton, torch.float64, E * self.nin, "skeleton"),
                                             _ptr(inflow, torch.float64, None, "inflow"),
                                             _ptr(mean, torch.float64, E * self.nm, "mean")), self._h)

    def elrt_recover_radiance(self, nx, nz, in2rad, f2u, skeleton, inflow, u):
        """u [E][nu] FP64 (rows k nm + i) = in2rad_K x_in(K) + f2u_K (f2u may be None)."""
        import torch
        E = nx * nz
        self._sync_stream()
        _check(_lib.elrt_recover_radiance(self._h, nx, nz, _ptr(in2rad, None, E * self.nu * self.nin, "in2rad"),
                                          _dt(in2rad), _ptr(f2u, torch.float64, E * self.nu, "f2u"),
                                          _ptr(skeleton, torch.float64, E * self.nin, "skeleton"),
                                          _ptr(inflow, torch.float64, None, "inflow"),
                                          _ptr(u, torch.float64, E * self.nu, "u")), self._h)

    def elrt_recover_mean(self, nx, nz, in2sol, skeleton, inflow, mean):
        import torch
        E = nx * nz
        self._sync_stream()
        _check(_lib.elrt_recover_mean(self._h, nx, nz, _ptr(in2sol, None, E * self.nm * self.nin, "in2sol"),
                                      _dt(in2sol), _ptr(skeleton, torch.float64, E * self.nin, "skeleton"),
                                      _ptr(inflow, torch.float64, None, "inflow"),
                                      _ptr(mean, torch.float64, E * self.nm, "mean")), self._h)


def _net_check(status, h):
    if status != 0:
        msg = _lib.elrt_net_last_error(h)
        raise ElrtError(status, msg.decode() if msg else "")


class Net:
    """An elrt_net: the element network of Sec. 2.4.1 (calls run on the current torch stream)."""

    def __init__(self, p, n_angles, n_hidden=4, width=1024, activation="gelu", seed=0, features="log", _handle=None):
        import torch
        if _handle is None:
            d = NetDesc(p, n_angles, n_hidden, width, 0 if activation == "gelu" else 1, seed,
                        0 if features == "log" else 1)
            h = C.c_void_p()
            _check(_lib.elrt_net_create(C.byref(h), C.byref(d), C.c_void_p(torch.cuda.current_stream().cuda_stream)))
        else:
            h = _handle
        self._h = h
        a, b, c, nl, npar = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int32(), C.c_int64()
        _lib.elrt_net_sizes(h, C.byref(a), C.byref(b), C.byref(c), C.byref(nl), C.byref(npar))
        self.n_feat, self.n_feat_pad, self.n_out, self.n_layers, self.n_params = a.value, b.value, c.value, nl.value, npar.value
        self.p, self.n_angles, self.width = p, n_angles, width
        self.nm = (p + 1) ** 2
        self.nin = 2 * (p + 1) * n_angles

    @classmethod
    def elrt_net_load(cls, path):
        """A network restored from a checkpoint written by elrt_net_save (current device and stream)."""
        import torch
        h = C.c_void_p()
        _check(_lib.elrt_net_load(C.byref(h), os.fsencode(path), C.c_void_p(torch.cuda.current_stream().cuda_stream)))
        info = elrt_net_file_info(path)
        return cls(info["p"], info["n_angles"], info["n_hidden"], info["width"],
                   "gelu" if info["activation"] == 0 else "elu", info["seed"],
                   "log" if info["features"] == 0 else "linear", _handle=h)

    def elrt_net_save(self, path):
        self._s()
        _net_check(_lib.elrt_net_save(self._h, os.fsencode(path)), self._h)

    def _s(self):
        import torch
        _lib.elrt_net_set_stream(self._h, C.c_void_p(torch.cuda.current_stream().cuda_stream))

    def close(self):
        if getattr(self, "_h", None):
            _lib.elrt_net_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def layer_shape(self, l):
        out = self.n_out if l == self.n_layers - 1 else self.width
        inp = self.n_feat_pad if l == 0 else self.width
        return out, inp

    def elrt_net_params(self, layer, what, value=None):
        """what: 'W', 'b', 'dW', 'db'.  Returns a host array, or writes `value` (W, b)."""
        code = {"W": 0, "b": 1, "dW": 2, "db": 3}[what]
        out, inp = self.layer_shape(layer)
        shape = (out, inp) if code in (0, 2) else (out,)
        if value is None:
            buf = np.zeros(shape, dtype=np.float32)
            _net_check(_lib.elrt_net_params(self._h, layer, code, 0, buf.ctypes.data), self._h)
            return buf
        buf = np.ascontiguousarray(np.asarray(value, dtype=np.float32).reshape(shape))
        _net_check(_lib.elrt_net_params(self._h, layer, code, 1, buf.ctypes.data), self._h)

    def elrt_net_forward(self, x, y):
        import torch
        self._s()
        n = x.shape[0]
        _net_check(_lib.elrt_net_forward(self._h, n, _ptr(x, torch.float32, n * self.n_feat_pad, "x"),
                                         _ptr(y, torch.float32, n * self.n_out, "y")), self._h)

    def elrt_net_train_step(self, x, t, lr=0.0):
        import torch
        self._s()
        n = x.shape[0]
        loss = C.c_float()
        _net_check(_lib.elrt_net_train_step(self._h, n, _ptr(x, torch.float32, n * self.n_feat_pad, "x"),
                                            _ptr(t, torch.float32, n * self.n_out, "t"), float(lr), C.byref(loss)),
                   self._h)
        return loss.value

    def elrt_net_fit(self, kappa, omega, h_elem, in2out, in2sol, epochs, batch, lr=1e-3, seed=0):
        import torch
        self._s()
        n = omega.numel()
        o = TrainOpts(epochs, batch, lr, 0.9, 0.999, 1e-8, seed)
        losses = np.zeros(epochs, dtype=np.float32)
        _net_check(_lib.elrt_net_fit(self._h, n, _ptr(kappa, torch.float64, n * self.nm, "kappa"),
                                     _ptr(omega, torch.float64, n, "omega"), _ptr(h_elem, torch.float64, n, "h_elem"),
                                     _ptr(in2out, torch.float32, n * self.nin * self.nin, "in2out"),
                                     _ptr(in2sol, torch.float32, n * self.nm * self.nin, "in2sol"), C.byref(o),
                                     losses.ctypes.data), self._h)
        return losses

    def elrt_net_infer(self, kappa, omega, h, in2out, in2sol, h_elem=None):
        import torch
        self._s()
        n = omega.numel()
        _net_check(_lib.elrt_net_infer(self._h, n, float(h), _ptr(h_elem, torch.float64, n, "h_elem"),
                                       _ptr(kappa, torch.float64, n * self.nm, "kappa"),
                                       _ptr(omega, torch.float64, n, "omega"),
                                       _ptr(in2out, torch.float32, n * self.nin * self.nin, "in2out"),
                                       _ptr(in2sol, torch.float32, n * self.nm * self.nin, "in2sol")), self._h)


def elrt_net_file_info(path):
    """Description, standardisation flag, Adam step and value count of a network checkpoint, validated
    (header, size, CRC) on the host; raises ElrtError(EINVAL) on a bad file."""
    d, st, step, nv = NetDesc(), C.c_int32(), C.c_int64(), C.c_int64()
    _check(_lib.elrt_net_file_info(os.fsencode(path), C.byref(d), C.byref(st), C.byref(step), C.byref(nv)))
    return {"p": d.p, "n_angles": d.n_angles, "n_hidden": d.n_hidden, "width": d.width, "activation": d.activation,
            "seed": d.seed, "features": d.features, "standardised": st.value, "adam_step": step.value,
            "n_values": nv.value}


def elrt_build_local_learned(ctx, net, kappa, omega, h, in2out, in2sol, tol=1e-3, h_elem=None, estimate=None):
    """Learned operators with the energy-balance estimate and classical fallback; returns the
    number of elements re-solved classically."""
    import torch
    ctx._sync_stream()
    net._s()
    n = omega.numel()
    nf = C.c_int64()
    _check(_lib.elrt_build_local_learned(
        ctx._h, net._h, n, float(h), _ptr(h_elem, torch.float64, n, "h_elem"),
        _ptr(kappa, torch.float64, n * ctx.nm, "kappa"), _ptr(omega, torch.float64, n, "omega"), float(tol),
        _ptr(in2out, torch.float32, n * ctx.nin * ctx.nin, "in2out"),
        _ptr(in2sol, torch.float32, n * ctx.nm * ctx.nin, "in2sol"),
        _ptr(estimate, torch.float32, n, "estimate"), C.byref(nf)), ctx._h)
    return nf.value


def _field(ctx, nx, nz, h, kappa, omega, inflow):
    import torch
    E = nx * nz
    return Field(int(nx), int(nz), float(h), _ptr(kappa, torch.float64, E * ctx.nm, "kappa"),
                 _ptr(omega, torch.float64, E, "omega"),
                 _ptr(inflow, torch.float64, 2 * (nx + nz) * (ctx.p + 1) * (ctx.n_angles // 2), "inflow"))


def _opts(mode, refine_steps, rtol, max_iter, restart, net, learned_tol):
    return SolveOpts(int(mode), int(refine_steps), float(rtol), int(max_iter), int(restart),
                     net._h if net is not None else None, float(learned_tol))


def elrt_solve_batch(ctxs, fields, field_ctx, means, mode=LOCAL_FP32_IR, refine_steps=1, rtol=1e-8, max_iter=20000,
                     restart=12, net=None, learned_tol=1e-3, wave_bytes=0, workers=0):
    """Many uneven fields: fields[f] = (nx, nz, h, kappa, omega, inflow) tensors; field_ctx[f] indexes ctxs.
    Returns the per-field FieldStats."""
    import torch
    for c in ctxs:
        c._sync_stream()
    n = len(fields)
    F = (Field * max(n, 1))(*[_field(ctxs[field_ctx[i]], *fields[i]) for i in range(n)])
    fc = (C.c_int32 * max(n, 1))(*field_ctx)
    hs = (C.c_void_p * len(ctxs))(*[c._h.value for c in ctxs])
    ms = (C.c_void_p * max(n, 1))(*[_ptr(means[i], torch.float64, None, "mean") for i in range(n)])
    st = (FieldStats * max(n, 1))()
    o = _opts(mode, refine_steps, rtol, max_iter, restart, net, learned_tol)
    _check(_lib.elrt_solve_batch(hs, len(ctxs), F, fc, n, C.byref(o), int(wave_bytes), int(workers), ms, st))
    return list(st)[:n]
