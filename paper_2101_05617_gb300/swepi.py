"""Thin ctypes binding of libswepi.so (C ABI in include/swepi.h).

Argument marshalling only: every step of the numerical path runs in the
library's CUDA kernels.  Device vectors are torch float64 CUDA tensors
(contiguous, canonical layout [var][panel][e2][e1][k2][k1]); streams are torch
streams.  The functions keep the C names (sw_init, sw_rhs, sw_jvp,
sw_kiops_phi, sw_epi_step, ...); the class ``SWContext`` bundles them.

There is no fallback: if the library is missing or fails to load, importing
or calling raises.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# SWEPI_CHECKED=1 loads the bounds-checked build instead (libswepi_check.so, from
# build.build(checked=True); see sw_check_status)
CHECKED = os.environ.get("SWEPI_CHECKED") == "1"
LIB_PATH = os.path.join(_HERE, "libswepi_check.so" if CHECKED else "libswepi.so")

SW_OK = 0
STATUS = {0: "ok", -1: "invalid argument", -2: "out of memory", -3: "CUDA error",
          -4: "Krylov solver limit", -5: "device wait timed out", -6: "non-finite value",
          -7: "grid larger than the fixed scratch of sw_jvp_static_scratch"}


class SWError(RuntimeError):
    def __init__(self, call, status):
        super().__init__(f"{call} failed: {STATUS.get(status, status)} ({status})")
        self.status = status


class sw_params(ctypes.Structure):
    _fields_ = [("radius", ctypes.c_double), ("gravity", ctypes.c_double), ("omega", ctypes.c_double),
                ("lambda0", ctypes.c_double), ("phi0", ctypes.c_double), ("alpha0", ctypes.c_double),
                ("precision", ctypes.c_int)]


class sw_kiops_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("m_init", ctypes.c_int), ("m_min", ctypes.c_int),
                ("m_max", ctypes.c_int), ("iop", ctypes.c_int), ("tau_init", ctypes.c_double)]


class sw_profile_stats(ctypes.Structure):
    _fields_ = [("count", ctypes.c_longlong * 7), ("ms", ctypes.c_double * 7)]

    KINDS = ("face_jvp", "volume_jvp", "face_rhs", "volume_rhs", "expm", "linearize", "orthogonalisation")

    def as_dict(self):
        return {k: {"count": int(self.count[i]), "ms": float(self.ms[i])} for i, k in enumerate(self.KINDS)}


class sw_kiops_stats(ctypes.Structure):
    _fields_ = [("substeps", ctypes.c_int), ("rejects", ctypes.c_int), ("krylov_iters", ctypes.c_int),
                ("m_final", ctypes.c_int), ("tau_final", ctypes.c_double), ("err_last", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class sw_ens_tiles(ctypes.Structure):
    _fields_ = [("face_pts", ctypes.c_int), ("vol_tiles", ctypes.c_int), ("vec_len", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class sw_ens_stats(ctypes.Structure):
    _fields_ = [("ticks", ctypes.c_longlong), ("reads", ctypes.c_longlong), ("expm_batches", ctypes.c_longlong),
                ("launches", ctypes.c_longlong), ("iter_ms", ctypes.c_double), ("block", ctypes.c_int),
                ("ctas", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    """Load libswepi.so (raises if it is missing: there is no CPU fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        how = "paper_2101_05617_gb300.build.build(checked=True)" if CHECKED else "__graft_entry__.build()"
        raise ImportError(f"{os.path.basename(LIB_PATH)} not built ({LIB_PATH}); run {how}")
    L = ctypes.CDLL(LIB_PATH)
    vp, dp, ip, ll = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_longlong
    L.sw_init.argtypes = [ip, ip, ctypes.POINTER(sw_params), ctypes.POINTER(vp)]
    L.sw_free.argtypes = [vp]
    L.sw_free.restype = None
    L.sw_num_unknowns.argtypes = [vp]
    L.sw_num_unknowns.restype = ll
    L.sw_grid_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), dp]
    L.sw_node_xyz.argtypes = [vp, vp]
    L.sw_state_from_fields.argtypes = [vp, vp, vp, vp, vp]
    L.sw_set_bottom.argtypes = [vp, vp]
    L.sw_set_bottom_host.argtypes = [vp, vp]
    L.sw_rhs.argtypes = [vp, vp, vp, vp]
    L.sw_jvp.argtypes = [vp, vp, vp, ctypes.c_double, vp, vp]
    L.sw_jvp_static_scratch.argtypes = [vp, vp, vp, ctypes.c_double, vp, vp]
    L.sw_linearize.argtypes = [vp, vp, vp]
    L.sw_jvp_linearized.argtypes = [vp, vp, vp, vp]
    L.sw_set_jvp_mode.argtypes = [vp, ip]
    L.sw_set_kiops_driver.argtypes = [vp, ip]
    L.sw_set_orth_fused.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_int)]
    L.sw_kiops_phi.argtypes = [vp, vp, ctypes.c_double, ctypes.c_double, ip, ctypes.POINTER(vp),
                               ctypes.POINTER(sw_kiops_opts), vp, ctypes.POINTER(sw_kiops_stats), vp]
    L.sw_epi_step.argtypes = [vp, ip, ctypes.c_double, vp, ctypes.POINTER(sw_kiops_opts),
                              ctypes.POINTER(sw_kiops_stats), vp]
    L.sw_epi_step_host.argtypes = [vp, ip, ctypes.c_double, vp, ctypes.POINTER(sw_kiops_opts),
                                   ctypes.POINTER(sw_kiops_stats), vp]
    L.sw_epi_set_history.argtypes = [vp, ip, vp, vp, vp]
    L.sw_epi_coefficients.argtypes = [ip, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), dp]
    L.sw_dfr_operators.argtypes = [ip, dp, dp, dp, dp, dp]
    L.sw_node_coefficients.argtypes = [ctypes.POINTER(sw_params), ip, ip, dp, dp, dp]
    ipp = ctypes.POINTER(ctypes.c_int)
    L.sw_interface_transform.argtypes = [ip, ctypes.c_double, ipp, ipp, ipp, ipp, ipp, dp]
    L.sw_epi_reset.argtypes = [vp]
    L.sw_epi_checkpoint_size.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
    L.sw_epi_checkpoint_save.argtypes = [vp, vp, ctypes.c_size_t, vp]
    L.sw_epi_checkpoint_load.argtypes = [vp, vp, ctypes.c_size_t, vp]
    L.sw_kernel_launches.argtypes = [vp]
    L.sw_kernel_launches.restype = ll
    L.sw_profile.argtypes = [vp, ip]
    L.sw_profile_kinds.argtypes = [vp, ctypes.c_uint]
    L.sw_profile_every.argtypes = [vp, ip]
    L.sw_check_status.argtypes = [ctypes.POINTER(ctypes.c_int)]
    L.sw_check_inject.argtypes = [vp, ip]
    L.sw_profile_read.argtypes = [vp, ctypes.POINTER(sw_profile_stats)]
    L.sw_fp64_fma_peak.argtypes = [dp]
    fp = ctypes.POINTER(ctypes.c_float)
    L.sw_mlp_create.argtypes = [ctypes.POINTER(vp)]
    L.sw_mlp_free.argtypes = [vp]
    L.sw_mlp_free.restype = None
    L.sw_mlp_set_params.argtypes = [vp, vp, vp]
    L.sw_mlp_get_params.argtypes = [vp, vp, vp]
    L.sw_mlp_forward.argtypes = [vp, vp, ip, vp, vp]
    L.sw_mlp_gradient.argtypes = [vp, vp, vp, ip, vp, fp, vp]
    L.sw_mlp_train.argtypes = [vp, vp, vp, ip, ip, ctypes.c_float, vp, vp]
    L.sw_set_controller.argtypes = [vp, vp]
    L.sw_diagnostics.argtypes = [vp, vp, vp, vp, vp]
    L.sw_error_norms.argtypes = [vp, vp, vp, vp, vp]
    L.sw_kiops_log.argtypes = [vp, vp, ip]
    L.sw_kiops_log_clear.argtypes = [vp]
    L.sw_status_str.argtypes = [ip]
    L.sw_status_str.restype = ctypes.c_char_p
    L.sw_ens_create.argtypes = [ip, ctypes.POINTER(vp), ctypes.POINTER(vp)]
    L.sw_ens_free.argtypes = [vp]
    L.sw_ens_set_block.argtypes = [vp, ip]
    L.sw_ens_set_tiles.argtypes = [vp, ip, ctypes.POINTER(sw_ens_tiles)]
    L.sw_ens_get_tiles.argtypes = [vp, ip, ctypes.POINTER(sw_ens_tiles)]
    L.sw_ens_set_policy.argtypes = [vp, ctypes.c_double]
    L.sw_ens_tune.argtypes = [vp, ctypes.POINTER(vp), ip, ctypes.POINTER(ctypes.c_int), vp]
    L.sw_ens_epi_run.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_int), dp, ctypes.POINTER(vp),
                                 ctypes.POINTER(sw_kiops_opts), ctypes.POINTER(sw_kiops_stats), vp]
    L.sw_ens_stats_read.argtypes = [vp, ctypes.POINTER(sw_ens_stats)]
    L.sw_ens_profile.argtypes = [vp, ip]
    L.sw_ens_set_wait_test.argtypes = [vp, ctypes.c_double, ip]
    _lib = L
    return L


EXPORTED = ["sw_init", "sw_free", "sw_num_unknowns", "sw_grid_info", "sw_node_xyz", "sw_state_from_fields",
            "sw_set_bottom", "sw_set_bottom_host", "sw_rhs", "sw_jvp", "sw_jvp_static_scratch", "sw_linearize", "sw_jvp_linearized",
            "sw_set_jvp_mode", "sw_set_kiops_driver", "sw_set_orth_fused", "sw_kiops_phi", "sw_epi_step", "sw_epi_step_host", "sw_epi_set_history",
            "sw_epi_reset", "sw_epi_checkpoint_size", "sw_epi_checkpoint_save", "sw_epi_checkpoint_load",
            "sw_epi_coefficients", "sw_dfr_operators", "sw_node_coefficients",
            "sw_interface_transform", "sw_kernel_launches", "sw_profile", "sw_profile_kinds", "sw_profile_every", "sw_profile_read", "sw_check_status", "sw_check_inject", "sw_fp64_fma_peak",
            "sw_status_str", "sw_mlp_create", "sw_mlp_free", "sw_mlp_set_params", "sw_mlp_get_params",
            "sw_mlp_forward", "sw_mlp_gradient", "sw_mlp_train", "sw_set_controller", "sw_kiops_log",
            "sw_kiops_log_clear", "sw_diagnostics", "sw_error_norms", "sw_ens_create", "sw_ens_free",
            "sw_ens_set_block", "sw_ens_set_tiles", "sw_ens_get_tiles", "sw_ens_set_policy", "sw_ens_tune",
            "sw_ens_epi_run", "sw_ens_stats_read", "sw_ens_profile", "sw_ens_set_wait_test"]

MLP_PARAMS = 5378
MLP_NORM = 36
KIOPS_LOG_FIELDS = 23


def _check(call, rc):
    if rc != SW_OK:
        raise SWError(call, rc)


def _dev_ptr(t, n=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError("expected a contiguous float64 CUDA tensor")
    if n is not None and t.numel() < n:
        raise ValueError(f"tensor has {t.numel()} elements, need {n}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _host(a, n):
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    if a.size < n:
        raise ValueError("host array too small")
    return a


def make_opts(tol=1e-10, m_init=10, m_min=10, m_max=128, iop=2, tau_init=0.0):
    return sw_kiops_opts(tol, m_init, m_min, m_max, iop, tau_init)


# ------------------------------------------------------------------ C names
def sw_init(n_e, p, rotation=(0.0, 0.0, 0.0), radius=6.37122e6, gravity=9.80616, omega=7.292e-5, precision=0):
    """precision 0: FP64 throughout; 1: the complex64-bulk form from the start."""
    prm = sw_params(radius, gravity, omega, rotation[0], rotation[1], rotation[2], int(precision))
    h = ctypes.c_void_p()
    _check("sw_init", lib().sw_init(int(n_e), int(p), ctypes.byref(prm), ctypes.byref(h)))
    return h


def sw_free(ctx):
    lib().sw_free(ctx)


def sw_num_unknowns(ctx):
    return int(lib().sw_num_unknowns(ctx))


def sw_node_xyz(ctx):
    n = sw_num_unknowns(ctx)
    out = np.empty(n, dtype=np.float64)
    _check("sw_node_xyz", lib().sw_node_xyz(ctx, out.ctypes.data_as(ctypes.c_void_p)))
    return out.reshape(3, -1)


def sw_state_from_fields(ctx, h, hB, V):
    n = sw_num_unknowns(ctx)
    nodes = n // 3
    h, hB, V = _host(h, nodes), _host(hB, nodes), _host(V, n)
    q = np.empty(n, dtype=np.float64)
    _check("sw_state_from_fields", lib().sw_state_from_fields(
        ctx, h.ctypes.data_as(ctypes.c_void_p), hB.ctypes.data_as(ctypes.c_void_p),
        V.ctypes.data_as(ctypes.c_void_p), q.ctypes.data_as(ctypes.c_void_p)))
    return q


def sw_set_bottom(ctx, hB):
    """Bottom height at the nodes from a float64 CUDA tensor (the C call takes a device pointer)."""
    nodes = sw_num_unknowns(ctx) // 3
    _check("sw_set_bottom", lib().sw_set_bottom(ctx, _dev_ptr(hB, nodes)))


def sw_set_bottom_host(ctx, hB):
    nodes = sw_num_unknowns(ctx) // 3
    hB = _host(hB, nodes)
    _check("sw_set_bottom_host", lib().sw_set_bottom_host(ctx, hB.ctypes.data_as(ctypes.c_void_p)))


def sw_rhs(ctx, q, F, stream=None):
    n = sw_num_unknowns(ctx)
    _check("sw_rhs", lib().sw_rhs(ctx, _dev_ptr(q, n), _dev_ptr(F, n), _stream(stream)))


def sw_jvp(ctx, q, v, eps, Jv, stream=None):
    n = sw_num_unknowns(ctx)
    _check("sw_jvp", lib().sw_jvp(ctx, _dev_ptr(q, n), _dev_ptr(v, n), float(eps), _dev_ptr(Jv, n),
                                  _stream(stream)))


def sw_jvp_static_scratch(ctx, q, v, eps, Jv, stream=None):
    """sw_jvp for callers that may not allocate device memory while running;
    the interface-flux scratch is a fixed 16 MiB array inside the library."""
    n = sw_num_unknowns(ctx)
    _check("sw_jvp_static_scratch", lib().sw_jvp_static_scratch(ctx, _dev_ptr(q, n), _dev_ptr(v, n), float(eps),
                                                                _dev_ptr(Jv, n), _stream(stream)))


def sw_linearize(ctx, q, stream=None):
    n = sw_num_unknowns(ctx)
    _check("sw_linearize", lib().sw_linearize(ctx, _dev_ptr(q, n), _stream(stream)))


def sw_jvp_linearized(ctx, v, Jv, stream=None):
    n = sw_num_unknowns(ctx)
    _check("sw_jvp_linearized", lib().sw_jvp_linearized(ctx, _dev_ptr(v, n), _dev_ptr(Jv, n), _stream(stream)))


def sw_set_jvp_mode(ctx, mode):
    _check("sw_set_jvp_mode", lib().sw_set_jvp_mode(ctx, int(mode)))


def sw_set_orth_fused(ctx, enable):
    """Both orthogonalisation passes in one cooperative launch (1) or two (0);
    returns 1 when the next phi-function call will fuse them."""
    active = ctypes.c_int(0)
    _check("sw_set_orth_fused", lib().sw_set_orth_fused(ctx, int(enable), ctypes.byref(active)))
    return active.value


def sw_set_kiops_driver(ctx, driver):
    """0: the phi-function solver's controller on the host; 1: on the device (one CUDA graph per call)."""
    _check("sw_set_kiops_driver", lib().sw_set_kiops_driver(ctx, int(driver)))


def sw_kiops_phi(ctx, q_lin, dt, tau_out, b, w, opts=None, stream=None):
    n = sw_num_unknowns(ctx)
    ptrs = (ctypes.c_void_p * len(b))(*[None if x is None else _dev_ptr(x, n).value for x in b])
    st = sw_kiops_stats()
    o = opts if opts is not None else make_opts()
    _check("sw_kiops_phi", lib().sw_kiops_phi(ctx, _dev_ptr(q_lin, n), float(dt), float(tau_out), len(b), ptrs,
                                              ctypes.byref(o), _dev_ptr(w, n), ctypes.byref(st), _stream(stream)))
    return st.as_dict()


def sw_epi_step(ctx, order, dt, q, opts=None, stream=None):
    n = sw_num_unknowns(ctx)
    st = sw_kiops_stats()
    o = opts if opts is not None else make_opts()
    _check("sw_epi_step", lib().sw_epi_step(ctx, int(order), float(dt), _dev_ptr(q, n), ctypes.byref(o),
                                            ctypes.byref(st), _stream(stream)))
    return st.as_dict()


def _host_ptr(t, n):
    import torch
    if not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError("expected a contiguous float64 host tensor")
    if t.numel() < n:
        raise ValueError(f"tensor has {t.numel()} elements, need {n}")
    return ctypes.c_void_p(t.data_ptr())


def sw_epi_step_host(ctx, order, dt, q_host, opts=None, stream=None):
    """sw_epi_step on a host tensor (pinned or pageable), copied in and back by the library."""
    n = sw_num_unknowns(ctx)
    st = sw_kiops_stats()
    o = opts if opts is not None else make_opts()
    _check("sw_epi_step_host", lib().sw_epi_step_host(ctx, int(order), float(dt), _host_ptr(q_host, n),
                                                      ctypes.byref(o), ctypes.byref(st), _stream(stream)))
    return st.as_dict()


def sw_epi_coefficients(order):
    """The library's EPI coefficient matrix of `order` (M x P numpy array); host only."""
    M, P = ctypes.c_int(), ctypes.c_int()
    A = (ctypes.c_double * 16)()
    _check("sw_epi_coefficients", lib().sw_epi_coefficients(int(order), ctypes.byref(M), ctypes.byref(P), A))
    return np.array(A[:M.value * P.value]).reshape(M.value, P.value)


def sw_dfr_operators(p):
    """The library's DFR operators of degree p: (xi, w, D_ext, l_minus, l_plus); host only."""
    ns = int(p) + 1
    xi, w, lm, lp = (np.zeros(ns) for _ in range(4))
    D = np.zeros((ns, ns + 2))
    ptr = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))   # noqa: E731
    _check("sw_dfr_operators", lib().sw_dfr_operators(int(p), ptr(xi), ptr(w), ptr(D), ptr(lm), ptr(lp)))
    return xi, w, D, lm, lp


def sw_node_coefficients(rotation, panel, X, Y, radius=6.37122e6, gravity=9.80616, omega=7.292e-5):
    """The library's 13 node coefficients at points (X, Y) of a panel: [13, npts]; host only."""
    X = np.ascontiguousarray(X, dtype=np.float64).ravel()
    Y = np.ascontiguousarray(Y, dtype=np.float64).ravel()
    if X.size != Y.size:
        raise ValueError("X and Y differ in size")
    prm = sw_params(radius, gravity, omega, rotation[0], rotation[1], rotation[2], 0)
    out = np.zeros((13, X.size))
    ptr = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))   # noqa: E731
    _check("sw_node_coefficients", lib().sw_node_coefficients(ctypes.byref(prm), int(panel), X.size, ptr(X), ptr(Y),
                                                              ptr(out)))
    return out


def sw_interface_transform(k, t):
    """Interface k of the library: ((pa, ea, pb, eb, rev), T[2, 2] at along-edge coordinate t); host only."""
    v = [ctypes.c_int() for _ in range(5)]
    T = np.zeros(4)
    _check("sw_interface_transform", lib().sw_interface_transform(
        int(k), float(t), *[ctypes.byref(x) for x in v], T.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return tuple(x.value for x in v), T.reshape(2, 2)


def sw_epi_set_history(ctx, i, q, F=None, stream=None):
    n = sw_num_unknowns(ctx)
    _check("sw_epi_set_history", lib().sw_epi_set_history(ctx, int(i), _dev_ptr(q, n),
                                                          None if F is None else _dev_ptr(F, n), _stream(stream)))


def sw_epi_reset(ctx):
    _check("sw_epi_reset", lib().sw_epi_reset(ctx))


def sw_epi_checkpoint_size(ctx):
    nb = ctypes.c_size_t(0)
    _check("sw_epi_checkpoint_size", lib().sw_epi_checkpoint_size(ctx, ctypes.byref(nb)))
    return int(nb.value)


def sw_epi_checkpoint_save(ctx, stream=None):
    """The multistep state as a host byte array (sw_epi_checkpoint_save)."""
    buf = np.zeros(sw_epi_checkpoint_size(ctx), dtype=np.uint8)
    _check("sw_epi_checkpoint_save", lib().sw_epi_checkpoint_save(ctx, ctypes.c_void_p(buf.ctypes.data), buf.size,
                                                                  _stream(stream)))
    return buf


def sw_epi_checkpoint_load(ctx, buf, stream=None):
    buf = np.ascontiguousarray(np.frombuffer(bytes(buf), dtype=np.uint8) if not isinstance(buf, np.ndarray) else buf,
                               dtype=np.uint8).reshape(-1)
    _check("sw_epi_checkpoint_load", lib().sw_epi_checkpoint_load(ctx, ctypes.c_void_p(buf.ctypes.data), buf.size,
                                                                  _stream(stream)))


def sw_kernel_launches(ctx):
    return int(lib().sw_kernel_launches(ctx))


def sw_profile(ctx, enable=True):
    _check("sw_profile", lib().sw_profile(ctx, 1 if enable else 0))


def sw_profile_kinds(ctx, mask):
    _check("sw_profile_kinds", lib().sw_profile_kinds(ctx, int(mask)))


def sw_profile_every(ctx, every):
    _check("sw_profile_every", lib().sw_profile_every(ctx, int(every)))


def sw_check_status():
    """(first check code since the last call, 0 = none; whether the library is the checked build)."""
    checked = ctypes.c_int(0)
    rc = lib().sw_check_status(ctypes.byref(checked))
    if rc < 0:
        raise SWError("sw_check_status", rc)
    return rc, bool(checked.value)


def sw_check_inject(ctx, what):
    _check("sw_check_inject", lib().sw_check_inject(ctx, int(what)))


def sw_profile_read(ctx):
    st = sw_profile_stats()
    _check("sw_profile_read", lib().sw_profile_read(ctx, ctypes.byref(st)))
    return st.as_dict()


def sw_fp64_fma_peak():
    t = ctypes.c_double()
    _check("sw_fp64_fma_peak", lib().sw_fp64_fma_peak(ctypes.byref(t)))
    return t.value


def _f32_dev(t, n=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError("expected a contiguous float32 CUDA tensor")
    if n is not None and t.numel() < n:
        raise ValueError("tensor too small")
    return ctypes.c_void_p(t.data_ptr())


def sw_mlp_create():
    h = ctypes.c_void_p()
    _check("sw_mlp_create", lib().sw_mlp_create(ctypes.byref(h)))
    return h


def sw_mlp_free(m):
    lib().sw_mlp_free(m)


def sw_mlp_set_params(m, params=None, norm=None):
    pa = None if params is None else np.ascontiguousarray(params, dtype=np.float32)
    no = None if norm is None else np.ascontiguousarray(norm, dtype=np.float32)
    if pa is not None and pa.size != MLP_PARAMS or no is not None and no.size != MLP_NORM:
        raise ValueError("wrong parameter or normalisation size")
    _check("sw_mlp_set_params", lib().sw_mlp_set_params(
        m, None if pa is None else pa.ctypes.data_as(ctypes.c_void_p),
        None if no is None else no.ctypes.data_as(ctypes.c_void_p)))


def sw_mlp_get_params(m):
    master = np.empty(MLP_PARAMS, dtype=np.float32)
    bf16 = np.empty(MLP_PARAMS, dtype=np.float32)
    _check("sw_mlp_get_params", lib().sw_mlp_get_params(m, master.ctypes.data_as(ctypes.c_void_p),
                                                        bf16.ctypes.data_as(ctypes.c_void_p)))
    return master, bf16


def sw_mlp_forward(m, X, Y, stream=None):
    n = X.shape[0]
    _check("sw_mlp_forward", lib().sw_mlp_forward(m, _f32_dev(X, 16 * n), n, _f32_dev(Y, 2 * n), _stream(stream)))


def sw_mlp_gradient(m, X, T, stream=None):
    n = X.shape[0]
    g = np.empty(MLP_PARAMS, dtype=np.float32)
    loss = ctypes.c_float()
    _check("sw_mlp_gradient", lib().sw_mlp_gradient(m, _f32_dev(X, 16 * n), _f32_dev(T, 2 * n), n,
                                                    g.ctypes.data_as(ctypes.c_void_p), ctypes.byref(loss),
                                                    _stream(stream)))
    return g, loss.value


def sw_mlp_train(m, X, T, steps, lr, stream=None):
    n = X.shape[0]
    losses = np.empty(max(1, steps), dtype=np.float32)
    _check("sw_mlp_train", lib().sw_mlp_train(m, _f32_dev(X, 16 * n), _f32_dev(T, 2 * n), n, int(steps),
                                              float(lr), losses.ctypes.data_as(ctypes.c_void_p), _stream(stream)))
    return losses[:steps]


def sw_set_controller(ctx, m):
    _check("sw_set_controller", lib().sw_set_controller(ctx, m))


def sw_kiops_log(ctx):
    have = lib().sw_kiops_log(ctx, None, 0)
    if have < 0:
        raise SWError("sw_kiops_log", have)
    out = np.empty(max(1, have) * KIOPS_LOG_FIELDS, dtype=np.float32)
    got = lib().sw_kiops_log(ctx, out.ctypes.data_as(ctypes.c_void_p), have)
    if got < 0:
        raise SWError("sw_kiops_log", got)
    return out[:have * KIOPS_LOG_FIELDS].reshape(have, KIOPS_LOG_FIELDS)


def sw_kiops_log_clear(ctx):
    _check("sw_kiops_log_clear", lib().sw_kiops_log_clear(ctx))


def sw_diagnostics(ctx, q, zeta=None, stream=None):
    """(mass, energy, potential enstrophy, max |zeta|) of Sec. 5."""
    n = sw_num_unknowns(ctx)
    out = np.empty(4, dtype=np.float64)
    z = None if zeta is None else _dev_ptr(zeta, n // 3)
    _check("sw_diagnostics", lib().sw_diagnostics(ctx, _dev_ptr(q, n), out.ctypes.data_as(ctypes.c_void_p), z,
                                                  _stream(stream)))
    return out


def sw_error_norms(ctx, q, q_ref, stream=None):
    n = sw_num_unknowns(ctx)
    out = np.empty(3, dtype=np.float64)
    _check("sw_error_norms", lib().sw_error_norms(ctx, _dev_ptr(q, n), _dev_ptr(q_ref, n),
                                                  out.ctypes.data_as(ctypes.c_void_p), _stream(stream)))
    return out


def sw_status_str(status):
    return lib().sw_status_str(int(status)).decode()


def sw_ens_create(ctxs):
    arr = (ctypes.c_void_p * len(ctxs))(*[c for c in ctxs])
    e = ctypes.c_void_p()
    _check("sw_ens_create", lib().sw_ens_create(len(ctxs), arr, ctypes.byref(e)))
    return e


def sw_ens_free(e):
    _check("sw_ens_free", lib().sw_ens_free(e))


def sw_ens_set_block(e, block):
    _check("sw_ens_set_block", lib().sw_ens_set_block(e, int(block)))


def sw_ens_set_tiles(e, member, face_pts, vol_tiles, vec_len):
    t = sw_ens_tiles(int(face_pts), int(vol_tiles), int(vec_len))
    _check("sw_ens_set_tiles", lib().sw_ens_set_tiles(e, int(member), ctypes.byref(t)))


def sw_ens_get_tiles(e, member):
    t = sw_ens_tiles()
    _check("sw_ens_get_tiles", lib().sw_ens_get_tiles(e, int(member), ctypes.byref(t)))
    return t.as_dict()


def sw_ens_set_policy(e, theta):
    _check("sw_ens_set_policy", lib().sw_ens_set_policy(e, float(theta)))


def _ptr_array(qs, sizes):
    return (ctypes.c_void_p * len(qs))(*[_dev_ptr(q, n).value for q, n in zip(qs, sizes)])


def sw_ens_tune(e, qs, sizes, iters=8, stream=None):
    blk = ctypes.c_int(0)
    _check("sw_ens_tune", lib().sw_ens_tune(e, _ptr_array(qs, sizes), int(iters), ctypes.byref(blk),
                                            _stream(stream)))
    return blk.value


def sw_ens_epi_run(e, steps, orders, dts, qs, sizes, opts=None, stream=None):
    k = len(qs)
    o = opts if opts is not None else make_opts()
    ords = (ctypes.c_int * k)(*[int(x) for x in orders])
    dtv = np.ascontiguousarray(dts, dtype=np.float64).reshape(-1)
    if dtv.size != k or len(orders) != k:
        raise ValueError("one order and one dt per member")
    st = (sw_kiops_stats * k)()
    _check("sw_ens_epi_run", lib().sw_ens_epi_run(e, int(steps), ords, dtv.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                                  _ptr_array(qs, sizes), ctypes.byref(o), st, _stream(stream)))
    return [st[i].as_dict() for i in range(k)]


def sw_ens_profile(e, enable=True):
    _check("sw_ens_profile", lib().sw_ens_profile(e, int(bool(enable))))


def sw_ens_set_wait_test(e, limit_s, extra):
    _check("sw_ens_set_wait_test", lib().sw_ens_set_wait_test(e, float(limit_s), int(extra)))


def sw_ens_stats_read(e):
    st = sw_ens_stats()
    _check("sw_ens_stats_read", lib().sw_ens_stats_read(e, ctypes.byref(st)))
    return st.as_dict()


class SWEnsemble:
    """A batched ensemble over existing SWContext members (kept alive here)."""

    def __init__(self, members):
        self.members = list(members)
        self.handle = sw_ens_create([m.handle for m in self.members])

    def close(self):
        if self.handle:
            sw_ens_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_block(self, block):
        sw_ens_set_block(self.handle, block)

    def set_tiles(self, member, face_pts, vol_tiles, vec_len):
        sw_ens_set_tiles(self.handle, member, face_pts, vol_tiles, vec_len)

    def tiles(self, member):
        return sw_ens_get_tiles(self.handle, member)

    def set_policy(self, theta):
        sw_ens_set_policy(self.handle, theta)

    def tune(self, qs, iters=8, stream=None):
        return sw_ens_tune(self.handle, qs, [m.n for m in self.members], iters, stream)

    def epi_run(self, steps, orders, dts, qs, stream=None, **opts):
        return sw_ens_epi_run(self.handle, steps, orders, dts, qs, [m.n for m in self.members], make_opts(**opts),
                              stream)

    def stats(self):
        return sw_ens_stats_read(self.handle)

    def profile(self, enable=True):
        sw_ens_profile(self.handle, enable)

    def set_wait_test(self, limit_s, extra):
        sw_ens_set_wait_test(self.handle, limit_s, extra)


class SWContext:
    """Owns one library context (grid + workspace) on the current CUDA device."""

    def __init__(self, n_e, p, rotation=(0.0, 0.0, 0.0), **consts):
        self.handle = sw_init(n_e, p, rotation, **consts)
        self.ne, self.p, self.ns = n_e, p, p + 1
        self.n = sw_num_unknowns(self.handle)
        self.nodes = self.n // 3

    def close(self):
        if self.handle:
            sw_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def node_xyz(self):
        return sw_node_xyz(self.handle)

    def state_from_fields(self, h, hB, V):
        return sw_state_from_fields(self.handle, h, hB, V)

    def set_bottom(self, hB):
        """hB: a float64 CUDA tensor (sw_set_bottom) or a host array (sw_set_bottom_host)."""
        import torch
        if isinstance(hB, torch.Tensor) and hB.is_cuda:
            sw_set_bottom(self.handle, hB)
        else:
            sw_set_bottom_host(self.handle, np.asarray(hB))

    def rhs(self, q, out=None, stream=None):
        import torch
        out = torch.empty_like(q) if out is None else out
        sw_rhs(self.handle, q, out, stream)
        return out

    def jvp(self, q, v, eps=1e-30, out=None, stream=None):
        import torch
        out = torch.empty_like(q) if out is None else out
        sw_jvp(self.handle, q, v, eps, out, stream)
        return out

    def linearize(self, q, stream=None):
        sw_linearize(self.handle, q, stream)

    def jvp_linearized(self, v, out=None, stream=None):
        import torch
        out = torch.empty_like(v) if out is None else out
        sw_jvp_linearized(self.handle, v, out, stream)
        return out

    def set_jvp_mode(self, mode):
        sw_set_jvp_mode(self.handle, mode)

    def set_kiops_driver(self, driver):
        sw_set_kiops_driver(self.handle, driver)

    def set_orth_fused(self, enable):
        return sw_set_orth_fused(self.handle, enable)

    def kiops_phi(self, q_lin, dt, b, tau_out=1.0, out=None, stream=None, **opts):
        import torch
        out = torch.empty_like(q_lin) if out is None else out
        st = sw_kiops_phi(self.handle, q_lin, dt, tau_out, b, out, make_opts(**opts), stream)
        return out, st

    def epi_step(self, order, dt, q, stream=None, **opts):
        return sw_epi_step(self.handle, order, dt, q, make_opts(**opts), stream)

    def epi_step_host(self, order, dt, q_host, stream=None, **opts):
        return sw_epi_step_host(self.handle, order, dt, q_host, make_opts(**opts), stream)

    def epi_set_history(self, i, q, F=None, stream=None):
        sw_epi_set_history(self.handle, i, q, F, stream)

    def epi_reset(self):
        sw_epi_reset(self.handle)

    def epi_checkpoint(self, stream=None):
        """Host copy (uint8 array) of the multistep state: history pairs, KIOPS warm start, controller features."""
        return sw_epi_checkpoint_save(self.handle, stream)

    def epi_restore(self, buf, stream=None):
        sw_epi_checkpoint_load(self.handle, buf, stream)

    def diagnostics(self, q, zeta=None, stream=None):
        """(mass, energy, potential enstrophy, max |zeta|) of q (sw_diagnostics)."""
        return sw_diagnostics(self.handle, q, zeta, stream)

    def kernel_launches(self):
        return sw_kernel_launches(self.handle)

    def profile(self, enable=True):
        sw_profile(self.handle, enable)

    def profile_kinds(self, *kinds):
        """Time only the named kernel families (sw_profile_stats.KINDS)."""
        mask = 0
        for k in kinds:
            mask |= 1 << sw_profile_stats.KINDS.index(k)
        sw_profile_kinds(self.handle, mask)

    def profile_every(self, every):
        """Bracket only every `every`-th launch of each timed JVP/RHS kernel family."""
        sw_profile_every(self.handle, every)

    def profile_read(self):
        return sw_profile_read(self.handle)
