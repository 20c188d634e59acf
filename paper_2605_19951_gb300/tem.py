"""Thin ctypes binding of libtem.so (the C ABI in include/tem.h).

Only argument marshalling lives here: every step of the path runs in the
library's CUDA kernels.  Device arrays are torch CUDA tensors (float64,
contiguous); host arrays are numpy arrays.  If the library has not been built
the import of a function raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libtem.so")

TEM_OK = 0
TEM_FP64 = 0
TEM_FP32_REFINED = 1
ERRORS = {-1: "TEM_ERR_ARG", -2: "TEM_ERR_OOM", -3: "TEM_ERR_PIVOT", -4: "TEM_ERR_TIMEOUT",
          -5: "TEM_ERR_CUDA", -6: "TEM_ERR_STATE", -7: "TEM_ERR_MESH"}
KERNEL_CLASSES = {"update": 0, "panel": 1, "fwd": 2, "bwd": 3, "bwd_upd": 4, "extend_add": 5, "fwd21": 6,
                  "fwd_sb": 7, "bwd_sb": 8, "invert": 9,
                  "residual": 10, "refine_vec": 11, "jacobian": 12, "nodal": 13,
                  "nodal_rhs": 14, "nodal_sweep": 15, "nodal_apply": 16, "update_tc": 17}

# C declarations, in include/tem.h order: name -> (restype, argtypes)
_P = ctypes.c_void_p
_I32, _I64, _D = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
SIGNATURES = {
    "tem_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, _P]),
    "tem_destroy": (ctypes.c_int, [_P]),
    "tem_last_error": (ctypes.c_char_p, [_P]),
    "tem_mesh": (ctypes.c_int, [_P, _I64, _P, _I64, _P, _P, _P, _I32]),
    "tem_poles": (ctypes.c_int, [_P, _I32, _P, _I32, _P]),
    "tem_times": (ctypes.c_int, [_P, _I32, _P, _I32, _D, _D, _D, _P]),
    "tem_fit_poles": (ctypes.c_int, [_I32, _I32, _P, _I32, _D, _D, _D, _I32, _P, _P, _P]),
    "tem_sources": (ctypes.c_int, [_P, _I32, _P, _P, _I32, _P]),
    "tem_factor": (ctypes.c_int, [_P, _P]),
    "tem_forward": (ctypes.c_int, [_P, _P]),
    "tem_jvp": (ctypes.c_int, [_P, _P, _P]),
    "tem_jtvp": (ctypes.c_int, [_P, _P, _P]),
    "tem_lsqr": (ctypes.c_int, [_P, _P, _P, _P, _D, _I32, _P]),
    "tem_lsqr_noalloc": (ctypes.c_int, [_P, _P, _P, _P, _D, _I32, _P]),
    "tem_gn_eval": (ctypes.c_int, [_P, _P, _P, _P, _D, _P, _P, _P]),
    "tem_model_step": (ctypes.c_int, [_P, _P, _P, _D, _P]),
    "tem_set_amalgamation": (ctypes.c_int, [_P, _I32]),
    "tem_set_refine": (ctypes.c_int, [_P, _I32, _D, _D]),
    "tem_set_refine_adjoint": (ctypes.c_int, [_P, _I32]),
    "tem_batch": (ctypes.c_int, [_P, _I32, _I32, _P, _P, _P, _P]),
    "tem_set_async": (ctypes.c_int, [_P, ctypes.c_int]),
    "tem_status": (ctypes.c_int, [_P]),
    "tem_set_tc_fronts": (ctypes.c_int, [_P, ctypes.c_int]),
    "tem_set_wait_limit": (ctypes.c_int, [_P, ctypes.c_uint32, _D]),
    "tem_set_tensor_cores": (ctypes.c_int, [_P, ctypes.c_int]),
    "tem_set_nodal": (ctypes.c_int, [_P, ctypes.c_int]),
    "tem_set_profiling": (ctypes.c_int, [_P, ctypes.c_int]),
    "tem_kernel_time": (ctypes.c_int, [_P, ctypes.POINTER(_D), ctypes.POINTER(_I64)]),
    "tem_launch_count": (_I64, []),
    "tem_info": (ctypes.c_int, [_P, _P]),
    "tem_export_pattern": (ctypes.c_int, [_P, ctypes.POINTER(_I64), _P, _P, _P, _P]),
    "tem_export_forward": (ctypes.c_int, [_P, _P]),
    "tem_export_dofs": (ctypes.c_int, [_P, _P]),
    "tem_level_info": (ctypes.c_int, [_P, _P]),
}


class TemStats(ctypes.Structure):
    _fields_ = [("n_dof", _I64), ("n_tet", _I64), ("n_param", _I64), ("n_faces_reg", _I64),
                ("n_fronts", _I64), ("n_levels", _I64), ("nnz_a", _I64), ("nnz_l", _I64),
                ("flops_factor", _D), ("max_front", _I64), ("bytes_device", _I64),
                ("m", _I32), ("n_times", _I32), ("n_tx", _I32), ("n_rx", _I32),
                ("precision", _I32), ("refine_steps", _I32), ("last_pivot_front", _I32),
                ("min_pivot_abs", _D), ("nnz_l11", _I64), ("n_solve_launch", _I64),
                ("pole_solves", _I64), ("solve_calls", _I64), ("tc_ctas_per_sm", _I32), ("refine_steps_adjoint", _I32),
                ("tc_prod_launches", _I64), ("simt_prod_launches", _I64),
                ("n_nodes", _I64), ("nnz_l_nodal", _I64), ("nodal", _I32), ("reserved0", _I32),
                ("tc_update_launches", _I64)]


class TemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load():
    """Load libtem.so (built by paper_2605_19951_gb300.build); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libtem.so not built ({LIB_PATH}); run paper_2605_19951_gb300.build")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(ctx, code):
    if code != TEM_OK:
        msg = load().tem_last_error(ctx).decode(errors="replace")
        raise TemError(code, msg)


def _host(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(_P)


def _dev(t, n=None):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    if n is not None and t.numel() != n:
        raise ValueError(f"expected {n} elements, got {t.numel()}")
    return _P(t.data_ptr())


# -- C-ABI functions (same names) ------------------------------------------------

def tem_create(precision=TEM_FP32_REFINED, stream=None):
    lib = load()
    ctx = _P()
    sp = None if stream is None else _P(int(stream))
    code = lib.tem_create(ctypes.byref(ctx), precision, sp)
    if code != TEM_OK:
        raise TemError(code, lib.tem_last_error(None).decode(errors="replace"))
    return ctx


def tem_destroy(ctx):
    return load().tem_destroy(ctx)


def tem_mesh(ctx, xyz, tets, sigma, is_param, leaf_max=0):
    x, px = _host(xyz, np.float64)
    t, pt = _host(tets, np.int32)
    s, ps = _host(sigma, np.float64)
    m, pm = _host(is_param, np.uint8)
    _check(ctx, load().tem_mesh(ctx, x.shape[0], px, t.shape[0], pt, ps, pm, int(leaf_max)))


def tem_poles(ctx, xi, alpha):
    xi = np.asarray(xi, dtype=np.complex128)
    alpha = np.asarray(alpha, dtype=np.complex128)
    a, pa = _host(np.stack([xi.real, xi.imag], axis=-1), np.float64)
    b, pb = _host(np.stack([alpha.real, alpha.imag], axis=-1), np.float64)
    _check(ctx, load().tem_poles(ctx, xi.shape[0], pa, alpha.shape[1], pb))


def tem_times(ctx, times, n_z=2200, z_min=1e-2, z_max=1e9, mu=1e-4):
    """Fit the residues alpha_i^[j] of the context's poles for new observation
    times on the device (penalised least squares over {0} and n_z log-spaced
    z in [z_min, z_max]); returns them as complex [m, K]."""
    t, pt = _host(times, np.float64)
    m = tem_info(ctx)["m"]
    out = np.zeros((m, t.shape[0], 2))
    _check(ctx, load().tem_times(ctx, t.shape[0], pt, int(n_z), float(z_min), float(z_max), float(mu),
                                 out.ctypes.data_as(_P)))
    return out[..., 0] + 1j * out[..., 1]


def tem_fit_poles(xi0, times, n_z=2200, z_min=1e-2, z_max=1e9, mu=1e-4, max_iter=300, stream=None):
    """Poles fitted on the device by variable projection from the starting
    poles xi0 (complex, Re < 0 < Im) for the fitting times; returns
    (poles, (f_start, f_end, steps))."""
    xi0 = np.asarray(xi0, dtype=np.complex128)
    x = np.ascontiguousarray(np.stack([xi0.real, xi0.imag], axis=-1), dtype=np.float64)
    t, pt = _host(times, np.float64)
    obj = np.zeros(3)
    code = load().tem_fit_poles(xi0.shape[0], t.shape[0], pt, int(n_z), float(z_min), float(z_max), float(mu),
                                int(max_iter), x.ctypes.data_as(_P), obj.ctypes.data_as(_P),
                                None if stream is None else _P(int(stream)))
    _check(None, code)
    return x[:, 0] + 1j * x[:, 1], tuple(obj)


def tem_sources(ctx, loops, rx):
    ptr = np.zeros(len(loops) + 1, dtype=np.int64)
    ptr[1:] = np.cumsum([len(lp) for lp in loops])
    verts = np.concatenate([np.asarray(lp, dtype=np.int32) for lp in loops])
    p, pp = _host(ptr, np.int64)
    v, pv = _host(verts, np.int32)
    r, pr = _host(rx, np.float64)
    _check(ctx, load().tem_sources(ctx, len(loops), pp, pv, r.shape[0], pr))


def tem_factor(ctx, log_sigma):
    _check(ctx, load().tem_factor(ctx, _dev(log_sigma)))


def tem_forward(ctx, d):
    _check(ctx, load().tem_forward(ctx, _dev(d)))


def tem_jvp(ctx, v, jv):
    _check(ctx, load().tem_jvp(ctx, _dev(v), _dev(jv)))


def tem_jtvp(ctx, w, jtw):
    _check(ctx, load().tem_jtvp(ctx, _dev(w), _dev(jtw)))


def tem_lsqr(ctx, d_obs, wd, m_ref, lam, n_iter, dm):
    _check(ctx, load().tem_lsqr(ctx, _dev(d_obs), _dev(wd), _dev(m_ref), float(lam), int(n_iter),
                                _dev(dm)))


def tem_lsqr_noalloc(ctx, d_obs, wd, m_ref, lam, n_iter, dm):
    """tem_lsqr with its work vectors in the library's fixed device array (no
    allocation); see include/tem.h for the size limit and sharing rules."""
    _check(ctx, load().tem_lsqr_noalloc(ctx, _dev(d_obs), _dev(wd), _dev(m_ref), float(lam), int(n_iter),
                                        _dev(dm)))


def tem_gn_eval(ctx, d_obs, wd, m_ref, lam, dm=None, grad=None):
    """(phi, data term, R, chi2, grad . dm) at the current model and data; fills grad if given."""
    out = np.zeros(5)
    _check(ctx, load().tem_gn_eval(ctx, _dev(d_obs), _dev(wd), _dev(m_ref), float(lam),
                                   None if dm is None else _dev(dm), None if grad is None else _dev(grad),
                                   out.ctypes.data_as(_P)))
    return out


def tem_model_step(ctx, m, dm, eta, out):
    _check(ctx, load().tem_model_step(ctx, _dev(m), _dev(dm), float(eta), _dev(out)))


def tem_set_refine(ctx, steps, floor_tau=1e-6, tol=0.0):
    _check(ctx, load().tem_set_refine(ctx, int(steps), float(floor_tau), float(tol)))


def tem_set_refine_adjoint(ctx, steps):
    _check(ctx, load().tem_set_refine_adjoint(ctx, int(steps)))


def tem_set_amalgamation(ctx, max_pivots):
    _check(ctx, load().tem_set_amalgamation(ctx, int(max_pivots)))


def tem_set_tensor_cores(ctx, enable):
    _check(ctx, load().tem_set_tensor_cores(ctx, int(bool(enable))))


TEM_BATCH_FACTOR, TEM_BATCH_FORWARD, TEM_BATCH_JTVP = 1, 2, 4


def tem_batch(ctxs, ops, log_sigma=None, d=None, w=None, jtw=None):
    """tem_batch over a list of contexts; the array lists match the contexts (None entries allowed)."""
    n = len(ctxs)
    arr = (_P * n)(*ctxs)

    def ptrs(ts):
        if ts is None:
            return None
        return (_P * n)(*[None if t is None else _dev(t).value for t in ts])

    code = load().tem_batch(arr, n, int(ops), ptrs(log_sigma), ptrs(d), ptrs(w), ptrs(jtw))
    if code != TEM_OK:
        raise TemError(code, load().tem_last_error(ctxs[0]).decode(errors="replace"))


def tem_set_async(ctx, enable):
    _check(ctx, load().tem_set_async(ctx, int(bool(enable))))


def tem_status(ctx):
    _check(ctx, load().tem_status(ctx))


def tem_set_tc_fronts(ctx, enable):
    _check(ctx, load().tem_set_tc_fronts(ctx, int(bool(enable))))


def tem_set_wait_limit(ctx, max_polls, max_seconds):
    _check(ctx, load().tem_set_wait_limit(ctx, int(max_polls), float(max_seconds)))


def tem_set_nodal(ctx, enable):
    _check(ctx, load().tem_set_nodal(ctx, int(bool(enable))))


def tem_set_profiling(ctx, kernel_class):
    kc = KERNEL_CLASSES.get(kernel_class, kernel_class) if kernel_class is not None else -1
    _check(ctx, load().tem_set_profiling(ctx, int(kc)))


def tem_kernel_time(ctx):
    ms, n = _D(), _I64()
    _check(ctx, load().tem_kernel_time(ctx, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def tem_launch_count():
    return int(load().tem_launch_count())


def tem_info(ctx):
    st = TemStats()
    _check(ctx, load().tem_info(ctx, ctypes.byref(st)))
    return {name: getattr(st, name) for name, _ in TemStats._fields_}


def tem_export_pattern(ctx, with_m=False):
    lib = load()
    nnz = _I64()
    _check(ctx, lib.tem_export_pattern(ctx, ctypes.byref(nnz), None, None, None, None))
    n = tem_info(ctx)["n_dof"]
    rp = np.zeros(n + 1, dtype=np.int64)
    ci = np.zeros(nnz.value, dtype=np.int32)
    kv = np.zeros(nnz.value)
    mv = np.zeros(nnz.value) if with_m else None
    _check(ctx, lib.tem_export_pattern(ctx, ctypes.byref(nnz), rp.ctypes.data_as(_P), ci.ctypes.data_as(_P),
                                       kv.ctypes.data_as(_P), mv.ctypes.data_as(_P) if with_m else None))
    return rp, ci, kv, mv


def tem_export_dofs(ctx):
    n = tem_info(ctx)["n_dof"]
    ev = np.zeros((n, 2), dtype=np.int64)
    _check(ctx, load().tem_export_dofs(ctx, ev.ctypes.data_as(_P)))
    return ev


def tem_level_info(ctx):
    """Per assembly-tree level: fronts, pivot-block entries, update-row entries, largest k."""
    out = np.zeros((tem_info(ctx)["n_levels"], 4), dtype=np.int64)
    _check(ctx, load().tem_level_info(ctx, out.ctypes.data_as(_P)))
    return out


def tem_export_forward(ctx):
    """Forward solutions g [m, N, n_tx] complex, library numbering."""
    info = tem_info(ctx)
    g = np.zeros((info["m"], info["n_dof"], info["n_tx"], 2))
    _check(ctx, load().tem_export_forward(ctx, g.ctypes.data_as(_P)))
    return g[..., 0] + 1j * g[..., 1]


# -- convenience wrapper ----------------------------------------------------------

class Model:
    """One survey on one GPU: mesh, poles, sources, and the current factors."""

    def __init__(self, xyz, tets, sigma, is_param, loops, rx, xi, alpha,
                 precision=TEM_FP32_REFINED, leaf_max=0, stream=None, amalgamation=None):
        import torch
        self.torch = torch
        self.ctx = tem_create(precision, stream)
        try:
            if amalgamation is not None:
                tem_set_amalgamation(self.ctx, amalgamation)
            tem_mesh(self.ctx, xyz, tets, sigma, is_param, leaf_max)
            tem_poles(self.ctx, xi, alpha)
            tem_sources(self.ctx, loops, rx)
        except Exception:
            tem_destroy(self.ctx)
            self.ctx = None
            raise
        info = tem_info(self.ctx)
        self.P = info["n_param"]
        self.shape = (info["n_tx"], info["n_rx"], info["n_times"])

    def close(self):
        if self.ctx is not None:
            tem_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _new(self, *shape):
        return self.torch.empty(*shape, dtype=self.torch.float64, device="cuda")

    def info(self):
        return tem_info(self.ctx)

    def factor(self, log_sigma):
        tem_factor(self.ctx, log_sigma.contiguous())

    def forward(self):
        d = self._new(*self.shape)
        tem_forward(self.ctx, d)
        return d

    def jvp(self, v):
        out = self._new(*self.shape)
        tem_jvp(self.ctx, v.contiguous(), out)
        return out

    def jtvp(self, w):
        out = self._new(self.P)
        tem_jtvp(self.ctx, w.contiguous(), out)
        return out

    def set_times(self, times, **fit):
        """New observation times: residues fitted on the device, factors kept
        (call forward() before jvp / jtvp / lsqr)."""
        alpha = tem_times(self.ctx, times, **fit)
        self.shape = (self.shape[0], self.shape[1], len(times))
        return alpha

    def lsqr(self, d_obs, wd, m_ref, lam, n_iter):
        dm = self._new(self.P)
        tem_lsqr(self.ctx, d_obs.contiguous(), wd.contiguous(), m_ref.contiguous(), lam, n_iter, dm)
        return dm


def _autograd_class():
    import torch

    class TemForward(torch.autograd.Function):
        """log-conductivity [P] -> data [n_tx, n_rx, K]; backward = J^T (Section 3.1).

        forward factors every shifted matrix and keeps the factors and the
        forward solutions g_i; backward reuses them (no per-time storage: the
        time dependence sits in the residues only).  A later forward on the
        same Model replaces the stored factors."""

        @staticmethod
        def forward(ctx, model, log_sigma):
            model.factor(log_sigma.detach())
            ctx.model = model
            return model.forward()

        @staticmethod
        def backward(ctx, grad_d):
            return None, ctx.model.jtvp(grad_d.contiguous())

    return TemForward


def __getattr__(name):
    if name == "TemForward":
        cls = _autograd_class()
        globals()["TemForward"] = cls
        return cls
    raise AttributeError(name)
