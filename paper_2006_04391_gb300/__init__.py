"""Python binding of the GB300 GSM library (``include/gsm.h``).

Argument marshalling only: every step of the material update and of the
basic scheme runs in the library's CUDA kernels (and cuFFT).  Tensors are
PyTorch CUDA tensors in structure-of-arrays layout ``[components, ld]``;
PyTorch provides device memory and streams.  There is no CPU fallback: if the
shared library has not been built, :func:`load` raises.

Names follow the C ABI: :func:`gsm_create`, :func:`gsm_update`,
:func:`gsm_destroy`, :func:`ms_create`, :func:`ms_run`, :func:`ms_solve`,
:func:`ms_destroy`, :func:`ms_workspace_bytes`.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libgsm_gb300.so")

GSM_OK, GSM_EINVAL, GSM_ENOMEM, GSM_ECUDA, GSM_ENOTCONV, GSM_ENOTSUP = 0, -1, -2, -3, -4, -5
GSM_PSI_ELASTIC, GSM_PSI_ELASTIC_VP_DEV, GSM_PSI_ELASTIC_VP_KIN = 0, 1, 2
GSM_PHI_NONE, GSM_PHI_NORTON, GSM_PHI_MS_FORCE = 0, 1, 2
GSM_FP64, GSM_FP32_FP64FIX, GSM_FP32 = 0, 1, 2
MS_PREC_FP64, MS_PREC_FP32_BULK = 0, 1
GSM_ODE23, GSM_ODE12, GSM_ODE23S = 0, 1, 2
ODE_METHODS = {"ode23": GSM_ODE23, "ode12": GSM_ODE12, "ode23s": GSM_ODE23S}

ST_CONVERGED, ST_NONFINITE, ST_CAP, ST_NOT_SPD = 1 << 16, 1 << 17, 1 << 18, 1 << 19

# Exported symbols declared in include/gsm.h.
EXPORTS = ("gsm_create", "gsm_destroy", "gsm_update", "gsm_strerror", "gsm_kernel_launches",
           "ms_create", "ms_destroy", "ms_workspace_bytes", "ms_run", "ms_solve", "ms_evaluate_noalloc",
           "serve_create", "serve_destroy", "serve_submit", "serve_tick", "serve_job_state", "serve_fetch",
           "serve_job_bytes", "ms_run_taped", "ms_adjoint", "ms_tape_destroy", "gsm_update_ode23",
           "gsm_update_ode", "gsm_update_host", "gsm_peak_probe")

_lib = None


class GsmError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = load().gsm_strerror(code).decode() if _lib is not None else str(code)
        super().__init__(f"{where}: {msg} ({code})")


class ms_problem(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("phase", ctypes.c_void_p), ("n_phases", ctypes.c_int),
                ("laws", ctypes.POINTER(ctypes.c_void_p)), ("precision", ctypes.c_int)]


class ms_load(ctypes.Structure):
    _fields_ = [("n_steps", ctypes.c_int), ("E", ctypes.POINTER(ctypes.c_double)),
                ("h", ctypes.POINTER(ctypes.c_double)), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("forced_iters", ctypes.POINTER(ctypes.c_int32)), ("switch_tol", ctypes.c_double),
                ("stress_mask", ctypes.c_int), ("Sigma", ctypes.POINTER(ctypes.c_double)), ("ref_update", ctypes.c_int),
                ("integrator", ctypes.c_int), ("ode_rtol", ctypes.c_double), ("ode_atol", ctypes.c_double),
                ("ode_max_substeps", ctypes.c_int)]


class ms_state(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_void_p), ("z", ctypes.c_void_p), ("resume", ctypes.c_int),
                ("E_prev", ctypes.c_double * 6)]


class serve_job(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("phase", ctypes.c_void_p), ("n_phases", ctypes.c_int),
                ("laws", ctypes.POINTER(ctypes.c_void_p)), ("precision", ctypes.c_int), ("n_steps", ctypes.c_int),
                ("E", ctypes.POINTER(ctypes.c_double)), ("h", ctypes.POINTER(ctypes.c_double)),
                ("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("switch_tol", ctypes.c_double),
                ("integrator", ctypes.c_int), ("ode_rtol", ctypes.c_double), ("ode_atol", ctypes.c_double),
                ("ode_max_substeps", ctypes.c_int)]


class ms_result(ctypes.Structure):
    _fields_ = [("Sigma", ctypes.POINTER(ctypes.c_double)), ("iters", ctypes.POINTER(ctypes.c_int32)),
                ("final_error", ctypes.POINTER(ctypes.c_double)),
                ("fp32_iters", ctypes.POINTER(ctypes.c_int32)), ("total_iters", ctypes.c_int64),
                ("E", ctypes.POINTER(ctypes.c_double)), ("reference", ctypes.POINTER(ctypes.c_double))]


def load(path=None):
    """Load the CUDA library (built by ``__graft_entry__.build()``); raises if missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    vp, i64, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
    lib.gsm_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, ctypes.POINTER(dbl),
                               ctypes.c_int, ctypes.c_int]
    lib.gsm_destroy.argtypes = [vp]
    lib.gsm_update.argtypes = [vp, i64, vp, vp, i64, dbl, vp, vp, vp, vp, vp]
    lib.gsm_update_ode23.argtypes = [vp, i64, vp, vp, vp, i64, dbl, dbl, dbl, ctypes.c_int, vp, vp, vp, vp, vp]
    lib.gsm_update_host.argtypes = [vp, i64, vp, vp, i64, dbl, vp, vp, vp, vp, i64, vp]
    lib.gsm_update_ode.argtypes = [vp, ctypes.c_int, i64, vp, vp, vp, i64, dbl, dbl, dbl, ctypes.c_int, vp, vp, vp, vp,
                                   vp]
    lib.gsm_strerror.restype = ctypes.c_char_p
    lib.gsm_strerror.argtypes = [ctypes.c_int]
    lib.gsm_kernel_launches.restype = i64
    lib.gsm_peak_probe.argtypes = [ctypes.c_int, i64, ctypes.c_int, ctypes.POINTER(dbl), vp]
    if hasattr(lib, "ms_evaluate_noalloc"):
        lib.ms_evaluate_noalloc.argtypes = [ctypes.c_int, vp, ctypes.c_int, ctypes.POINTER(vp), dbl, vp, vp, vp, vp,
                                            vp, vp]
    i32p, i64p, dblp = ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(dbl)
    if hasattr(lib, "serve_create"):
        lib.serve_create.argtypes = [ctypes.POINTER(vp), ctypes.c_size_t, ctypes.c_int, vp]
        lib.serve_destroy.argtypes = [vp]
        lib.serve_submit.argtypes = [vp, ctypes.POINTER(serve_job), i64p]
        lib.serve_tick.argtypes = [vp, i32p, i32p, i32p]
        lib.serve_job_state.argtypes = [vp, i64, i32p, i32p, i64p]
        lib.serve_fetch.argtypes = [vp, i64, dblp, i32p, dblp]
        lib.serve_job_bytes.argtypes = [ctypes.c_int, ctypes.c_int]
        lib.serve_job_bytes.restype = ctypes.c_size_t
    if hasattr(lib, "ms_run_taped"):
        lib.ms_run_taped.argtypes = [vp, ctypes.POINTER(ms_load), ctypes.POINTER(ms_result), ctypes.POINTER(vp)]
        lib.ms_adjoint.argtypes = [vp, dblp, ctypes.c_int, dbl, ctypes.c_int, dblp, i32p]
        lib.ms_tape_destroy.argtypes = [vp]
    for name in ("ms_create", "ms_destroy", "ms_run", "ms_solve", "ms_workspace_bytes"):
        if hasattr(lib, name):
            fn = getattr(lib, name)
            if name == "ms_create":
                fn.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(ms_problem), vp]
            elif name == "ms_destroy":
                fn.argtypes = [vp]
            elif name == "ms_run":
                fn.argtypes = [vp, ctypes.POINTER(ms_load), ctypes.POINTER(ms_state), ctypes.POINTER(ms_result)]
            elif name == "ms_solve":
                fn.argtypes = [ctypes.POINTER(ms_problem), ctypes.POINTER(ms_load), ctypes.POINTER(ms_state),
                               ctypes.POINTER(ms_result), vp]
            elif name == "ms_workspace_bytes":
                fn.argtypes = [ctypes.POINTER(ms_problem)]
                fn.restype = ctypes.c_size_t
    _lib = lib
    return lib


def _check(rc, where):
    if rc != GSM_OK:
        raise GsmError(rc, where)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def kernel_launches():
    return int(load().gsm_kernel_launches())


def peak_probe(precision, iters, blocks_per_sm=4, stream=None):
    """Launch the FMA-throughput probe (``gsm_peak_probe``); returns the number
    of FMAs the launch performs.  The caller times it on ``stream``."""
    f = ctypes.c_double()
    _check(load().gsm_peak_probe(int(precision), int(iters), int(blocks_per_sm), ctypes.byref(f),
                                 _stream_ptr(stream)), "gsm_peak_probe")
    return f.value


# ------------------------------------------------------------------ materials

class Material:
    """Owns a ``gsm_handle`` (see :func:`gsm_create`)."""

    def __init__(self, handle, psi_kind, phi_kind, params, precision):
        self.handle = handle
        self.psi_kind, self.phi_kind = psi_kind, phi_kind
        self.params, self.precision = tuple(params), precision

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.gsm_destroy(self.handle)
            self.handle = None


def gsm_create(psi_kind, phi_kind, params, precision=GSM_FP64):
    lib = load()
    h = ctypes.c_void_p()
    arr = (ctypes.c_double * len(params))(*[float(x) for x in params])
    _check(lib.gsm_create(ctypes.byref(h), psi_kind, phi_kind, arr, len(params), precision), "gsm_create")
    return Material(h, psi_kind, phi_kind, params, precision)


def norton(E, nu, sigma0, edot0, n, precision=GSM_FP64):
    return gsm_create(GSM_PSI_ELASTIC_VP_DEV, GSM_PHI_NORTON, (E, nu, sigma0, edot0, n), precision)


def elastic(E, nu, precision=GSM_FP64):
    return gsm_create(GSM_PSI_ELASTIC, GSM_PHI_NONE, (E, nu), precision)


def michel_suquet(E, nu, sigma_Y, H, edot0, sigma_d, n):
    """The paper's Michel-Suquet law (kinematic hardening H, yield sigma_Y); its
    internal variables are z (6) and alpha; integrated by gsm_update_ode23."""
    return gsm_create(GSM_PSI_ELASTIC_VP_KIN, GSM_PHI_MS_FORCE, (E, nu, sigma_Y, H, edot0, sigma_d, n))


def gsm_destroy(mat):
    if mat.handle:
        load().gsm_destroy(mat.handle)
        mat.handle = None


def gsm_update_ode23(mat, eps_n, eps, z_n, h, sigma, z, tangent=None, status=None, rtol=1e-3, atol=1e-6,
                     max_substeps=100000, stream=None, n_vox=None, method="ode23"):
    """Material update by ode23 (or, method="ode12", the Euler/Heun pair; method="ode23s",
    the Shampine-Reichelt Rosenbrock triple) over the
    load step (FP64 tensors ``[6, ld]``; internal variables ``[7, ld]`` (z,
    alpha) for the Michel-Suquet law; tangent ``[36, ld]`` = full
    dsigma/deps_{n+1} row-major; status ``[ld]``)."""
    lib = load()
    ld = eps.shape[1]
    n = ld if n_vox is None else int(n_vox)
    nz = 7 if mat.psi_kind == GSM_PSI_ELASTIC_VP_KIN else 6
    for t, rows in ((eps_n, 6), (eps, 6), (z_n, nz), (sigma, 6), (z, nz), (tangent, 36)):
        if t is not None and (t.dim() != 2 or t.shape[0] != rows or t.shape[1] != ld or not t.is_contiguous()):
            raise ValueError("fields must be contiguous [components, ld] tensors with a common ld")
    args = (n, _ptr(eps_n), _ptr(eps), _ptr(z_n), ld, float(h), float(rtol), float(atol), int(max_substeps),
            _ptr(sigma), _ptr(z), _ptr(tangent), _ptr(status), _stream_ptr(stream))
    if method == "ode23":
        rc = lib.gsm_update_ode23(mat.handle, *args)
    else:
        rc = lib.gsm_update_ode(mat.handle, ODE_METHODS[method], *args)
    _check(rc, "gsm_update_ode23")


def gsm_update(mat, eps, z_n, h, sigma, z, tangent=None, status=None, stream=None, n_vox=None):
    """Material update of ``n_vox`` voxels; tensors ``[6, ld]`` (tangent ``[21, ld]``, status ``[ld]``)."""
    lib = load()
    ld = eps.shape[1]
    n = ld if n_vox is None else int(n_vox)
    for t, rows in ((eps, 6), (z_n, 6), (sigma, 6), (z, 6), (tangent, 21)):
        if t is not None and (t.dim() != 2 or t.shape[0] != rows or t.shape[1] != ld or not t.is_contiguous()):
            raise ValueError("fields must be contiguous [components, ld] tensors with a common ld")
    rc = lib.gsm_update(mat.handle, n, _ptr(eps), _ptr(z_n), ld, float(h), _ptr(sigma), _ptr(z),
                        _ptr(tangent), _ptr(status), _stream_ptr(stream))
    _check(rc, "gsm_update")


def gsm_update_host(mat, eps, z_n, h, sigma, z, tangent=None, status=None, chunk=0, stream=None, n_vox=None):
    """gsm_update on pinned CPU tensors (``[6, ld]``, tangent ``[21, ld]``, status
    ``[ld]``), streamed through the device in chunks with copies overlapping the
    updates; asynchronous on ``stream``."""
    lib = load()
    ld = eps.shape[1]
    n = ld if n_vox is None else int(n_vox)
    for t, rows in ((eps, 6), (z_n, 6), (sigma, 6), (z, 6), (tangent, 21)):
        if t is not None and (t.dim() != 2 or t.shape[0] != rows or t.shape[1] != ld or not t.is_contiguous()):
            raise ValueError("fields must be contiguous [components, ld] tensors with a common ld")
    rc = lib.gsm_update_host(mat.handle, n, _ptr(eps), _ptr(z_n), ld, float(h), _ptr(sigma), _ptr(z), _ptr(tangent),
                             _ptr(status), int(chunk), _stream_ptr(stream))
    _check(rc, "gsm_update_host")


# -------------------------------------------------------------- basic scheme

class MsContext:
    def __init__(self, handle, N, laws, phase):
        self.handle, self.N, self.laws, self.phase = handle, N, laws, phase

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.ms_destroy(self.handle)
            self.handle = None


def _problem(phase, laws, precision):
    N = int(phase.shape[0])
    arr = (ctypes.c_void_p * len(laws))(*[m.handle.value for m in laws])
    prob = ms_problem(N, phase.data_ptr(), len(laws), ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p)), precision)
    return prob, arr


def ms_workspace_bytes(N, n_phases=2, precision=MS_PREC_FP64):
    lib = load()
    prob = ms_problem(int(N), None, int(n_phases), None, int(precision))
    return int(lib.ms_workspace_bytes(ctypes.byref(prob)))


def ms_create(phase, laws, precision=MS_PREC_FP64, stream=None):
    """Plan a basic-scheme solver; ``phase`` is a uint8 CUDA tensor (N, N, N)."""
    lib = load()
    prob, arr = _problem(phase, laws, precision)
    h = ctypes.c_void_p()
    _check(lib.ms_create(ctypes.byref(h), ctypes.byref(prob), _stream_ptr(stream)), "ms_create")
    ctx = MsContext(h, int(phase.shape[0]), list(laws), phase)
    ctx._arr = arr
    return ctx


def _mask_bits(stress_mask):
    if stress_mask is None:
        return 0
    if isinstance(stress_mask, (int, np.integer)):
        return int(stress_mask)
    return sum(1 << c for c, b in enumerate(stress_mask) if b)


def _load_struct(E, hs, tol, max_iter, forced_iters, switch_tol, stress_mask=None, Sigma=None, ref_update=False,
                 ode=None, ode_method="ode23"):
    E = np.ascontiguousarray(np.asarray(E, dtype=np.float64).reshape(-1, 6))
    hs = np.ascontiguousarray(np.asarray(hs, dtype=np.float64).reshape(-1))
    n = E.shape[0]
    if hs.shape[0] != n:
        raise ValueError("one step size per load step")
    f = None
    keep = [E, hs]
    if forced_iters is not None:
        f = np.ascontiguousarray(np.asarray(forced_iters, dtype=np.int32).reshape(-1))
        keep.append(f)
    S = None
    if Sigma is not None:
        S = np.ascontiguousarray(np.asarray(Sigma, dtype=np.float64).reshape(n, 6))
        keep.append(S)
    ld = ms_load(n, E.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                 hs.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(tol), int(max_iter),
                 f.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)) if f is not None else None, float(switch_tol),
                 _mask_bits(stress_mask), S.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if S is not None else None,
                 1 if ref_update else 0, 0 if ode is None else 1 + ODE_METHODS[ode_method],
                 float(ode[0]) if ode is not None else 1e-3, float(ode[1]) if ode is not None else 1e-6,
                 int(ode[2]) if ode is not None and len(ode) > 2 else 100000)
    return ld, keep, n


def _result_struct(n):
    out = {"Sigma": np.zeros((n, 6)), "iters": np.zeros(n, dtype=np.int32), "final_error": np.zeros(n),
           "fp32_iters": np.zeros(n, dtype=np.int32), "E": np.zeros((n, 6)), "reference": np.zeros((n, 2))}
    dp, ip = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)
    res = ms_result(out["Sigma"].ctypes.data_as(dp), out["iters"].ctypes.data_as(ip),
                    out["final_error"].ctypes.data_as(dp), out["fp32_iters"].ctypes.data_as(ip), 0,
                    out["E"].ctypes.data_as(dp), out["reference"].ctypes.data_as(dp))
    return res, out


def ms_run(ctx, E, hs, tol=1e-8, max_iter=10000, forced_iters=None, eps=None, z=None, resume=False,
           E_prev=None, switch_tol=0.0, check=True, stress_mask=None, Sigma=None, ref_update=False, ode=None,
           ode_method="ode23"):
    """Solve a load history.  Returns dict(Sigma, iters, final_error, fp32_iters, total_iters, E,
    reference, rc).  stress_mask: 6 booleans (or bits) of the macroscopic components whose stress
    (Sigma, default 0) is prescribed; ref_update: per-step reference medium from tangents;
    ode: None (implicit Euler) or (rtol, atol[, max_substeps]) for the update over each step by
    ode_method ("ode23", "ode12" or "ode23s")."""
    lib = load()
    ld, keep, n = _load_struct(E, hs, tol, max_iter, forced_iters, switch_tol, stress_mask, Sigma, ref_update,
                               ode, ode_method)
    res, out = _result_struct(n)
    st = None
    if eps is not None or z is not None:
        st = ms_state(eps.data_ptr(), z.data_ptr(), 1 if resume else 0,
                      (ctypes.c_double * 6)(*(E_prev if E_prev is not None else [0.0] * 6)))
    rc = lib.ms_run(ctx.handle, ctypes.byref(ld), ctypes.byref(st) if st is not None else None, ctypes.byref(res))
    if check and rc not in (GSM_OK, GSM_ENOTCONV):
        _check(rc, "ms_run")
    out["total_iters"] = int(res.total_iters)
    out["rc"] = rc
    return out


def ms_evaluate_noalloc(phase, laws, h, eps, z_n, sigma, z, mean, stream=None):
    """Allocation-free material evaluation of a phase field (see include/gsm.h).

    All tensors are caller-allocated CUDA tensors: ``eps``, ``z_n``, ``sigma``,
    ``z`` are [6, N^3] float64, ``mean`` is [6] float64."""
    lib = load()
    arr = (ctypes.c_void_p * len(laws))(*[m.handle.value for m in laws])
    rc = lib.ms_evaluate_noalloc(int(phase.shape[0]), phase.data_ptr(), len(laws),
                                 ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p)), float(h), _ptr(eps), _ptr(z_n),
                                 _ptr(sigma), _ptr(z), _ptr(mean), _stream_ptr(stream))
    _check(rc, "ms_evaluate_noalloc")


class Tape:
    """Checkpoints of a load history (``ms_run_taped``); keeps its context alive."""

    def __init__(self, handle, ctx, n_steps):
        self.handle, self.ctx, self.n_steps = handle, ctx, n_steps

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.ms_tape_destroy(self.handle)
            self.handle = None


def ms_run_taped(ctx, E, hs, tol=1e-10, max_iter=20000, forced_iters=None, ref_update=False):
    """Load history from a fresh state keeping per-step checkpoints; returns (result, Tape).
    ref_update: the forward run's per-step reference medium from tangents."""
    lib = load()
    ld, keep, n = _load_struct(E, hs, tol, max_iter, forced_iters, 0.0, ref_update=ref_update)
    res, out = _result_struct(n)
    th = ctypes.c_void_p()
    rc = lib.ms_run_taped(ctx.handle, ctypes.byref(ld), ctypes.byref(res), ctypes.byref(th))
    if rc not in (GSM_OK, GSM_ENOTCONV):
        _check(rc, "ms_run_taped")
    out["rc"] = rc
    return out, Tape(th, ctx, n)


def ms_adjoint(tape, w, phase_id=0, tol=1e-10, max_iter=20000, check=True):
    """dJ/d(E, sigma0, n) of a Norton phase for J = w . Sigma_K; returns (grad[3], lam_iters).

    With check=False a step that reached max_iter is not an error (the
    gradient of the capped solves is returned)."""
    lib = load()
    w = np.ascontiguousarray(np.asarray(w, dtype=np.float64).reshape(6))
    grad = np.zeros(3)
    its = np.zeros(tape.n_steps, dtype=np.int32)
    rc = lib.ms_adjoint(tape.handle, w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(phase_id),
                        float(tol), int(max_iter), grad.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                        its.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    if rc != GSM_OK and (check or rc != GSM_ENOTCONV):
        _check(rc, "ms_adjoint")
    return grad, its


def ms_destroy(ctx):
    if ctx.handle:
        load().ms_destroy(ctx.handle)
        ctx.handle = None


def ms_solve(phase, laws, E, hs, precision=MS_PREC_FP64, stream=None, **kw):
    """One-shot basic-scheme solve (ms_create + ms_run + ms_destroy)."""
    ctx = ms_create(phase, laws, precision, stream)
    try:
        return ms_run(ctx, E, hs, **kw)
    finally:
        ms_destroy(ctx)


# ------------------------------------------------------------------ serving

SERVE_QUEUED, SERVE_ACTIVE, SERVE_DONE, SERVE_DONE_NOTCONV = 0, 1, 2, 3


class Server:
    """A serving engine (``serve_create``): jobs are basic-scheme solves that
    are admitted by an HBM budget and advanced together, one batched
    iteration per :meth:`tick`."""

    def __init__(self, hbm_budget_bytes, max_active=64, stream=None):
        lib = load()
        self.handle = ctypes.c_void_p()
        _check(lib.serve_create(ctypes.byref(self.handle), int(hbm_budget_bytes), int(max_active),
                                _stream_ptr(stream)), "serve_create")
        self.n_steps = {}

    def submit(self, phase, laws, E, hs, tol=1e-6, max_iter=20000, precision=MS_PREC_FP32_BULK, switch_tol=0.0,
               ode=None, ode_method="ode23"):
        """Queue a job; ``phase`` is a host uint8 array (N, N, N).  ``ode`` = (rtol, atol[,
        max_substeps]) integrates the laws over each step by ``ode_method`` (FP64 jobs).
        Returns the job id."""
        lib = load()
        ph = np.ascontiguousarray(np.asarray(phase, dtype=np.uint8))
        E = np.ascontiguousarray(np.asarray(E, dtype=np.float64).reshape(-1, 6))
        hs = np.ascontiguousarray(np.asarray(hs, dtype=np.float64).reshape(-1))
        arr = (ctypes.c_void_p * len(laws))(*[m.handle.value for m in laws])
        job = serve_job(int(ph.shape[0]), ph.ctypes.data, len(laws), ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p)),
                        int(precision), E.shape[0], E.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                        hs.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(tol), int(max_iter),
                        float(switch_tol), 0 if ode is None else 1 + ODE_METHODS[ode_method],
                        float(ode[0]) if ode is not None else 1e-3, float(ode[1]) if ode is not None else 1e-6,
                        int(ode[2]) if ode is not None and len(ode) > 2 else 100000)
        jid = ctypes.c_int64()
        _check(lib.serve_submit(self.handle, ctypes.byref(job), ctypes.byref(jid)), "serve_submit")
        self.n_steps[jid.value] = E.shape[0]
        return jid.value

    def tick(self):
        """One batched iteration; returns (active, queued, finished) counts."""
        a, q, f = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(load().serve_tick(self.handle, ctypes.byref(a), ctypes.byref(q), ctypes.byref(f)), "serve_tick")
        return a.value, q.value, f.value

    def state(self, jid):
        st, step, it = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        _check(load().serve_job_state(self.handle, int(jid), ctypes.byref(st), ctypes.byref(step),
                                      ctypes.byref(it)), "serve_job_state")
        return st.value, step.value, it.value

    def fetch(self, jid):
        n = self.n_steps.pop(jid)
        Sigma = np.zeros((n, 6))
        iters = np.zeros(n, dtype=np.int32)
        ferr = np.zeros(n)
        rc = load().serve_fetch(self.handle, int(jid), Sigma.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                iters.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                ferr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        if rc not in (GSM_OK, GSM_ENOTCONV):
            _check(rc, "serve_fetch")
        return {"Sigma": Sigma, "iters": iters, "final_error": ferr, "rc": rc}

    def close(self):
        if getattr(self, "handle", None):
            load().serve_destroy(self.handle)
            self.handle = None

    def __del__(self):
        if _lib is not None:
            self.close()


def serve_job_bytes(N, precision=MS_PREC_FP32_BULK):
    return int(load().serve_job_bytes(int(N), int(precision)))


# ------------------------------------------------- differentiable homogenization

def _effective_stress_function():
    import torch

    class EffectiveStress(torch.autograd.Function):
        """Sigma_K(theta) for theta = (E, sigma0, n) of the Norton phase; the
        backward pass is the hand-written adjoint of the load history."""

        @staticmethod
        def forward(ctx, theta, phase, E_loads, hs, other_laws, nu, edot0, tol, adj_tol, precision):
            th = theta.detach().cpu().double().numpy()
            laws = [norton(float(th[0]), nu, float(th[1]), edot0, float(th[2]), precision=precision)]
            laws += [elastic(*p) for p in other_laws]
            mctx = ms_create(phase, laws, MS_PREC_FP64)
            res, tape = ms_run_taped(mctx, E_loads, hs, tol=tol)
            ctx.tape = tape
            ctx.adj_tol = adj_tol
            ctx.laws = laws
            return torch.tensor(res["Sigma"][-1], dtype=torch.float64)

        @staticmethod
        def backward(ctx, grad_out):
            grad, _ = ms_adjoint(ctx.tape, grad_out.detach().cpu().double().numpy(), 0, tol=ctx.adj_tol)
            return (torch.tensor(grad, dtype=torch.float64),) + (None,) * 9

    return EffectiveStress


_EFF = None


def effective_stress(theta, phase, E_loads, hs, inclusions=((400.0, 0.2),), nu=0.3, edot0=1.0, tol=1e-10,
                     adj_tol=1e-10, precision=GSM_FP64):
    """Differentiable final mean stress of a Norton-matrix composite.

    theta: float64 tensor (E, sigma0, n) of the matrix (phase id 0); phase:
    uint8 CUDA tensor (N, N, N) with ids 1.. for the elastic ``inclusions``.
    Returns Sigma_K (6,) whose backward pass runs ``ms_adjoint``."""
    global _EFF
    if _EFF is None:
        _EFF = _effective_stress_function()
    return _EFF.apply(theta, phase, E_loads, hs, tuple(inclusions), nu, edot0, tol, adj_tol, precision)
