"""ctypes wrappers around the C++ FP64 oracle (test infrastructure only).

Array layout is array-of-structs: ``eps[n, 6]``, ``z_n[n, 6]``.  Voigt order
(11, 22, 33, 23, 13, 12); strain-like vectors carry engineering shears,
stress-like vectors tensor shears (Sec. 3 of the paper: Voigt notation, and
H = diag(H,H,H,H/2,H/2,H/2) in Eq. michel_suquet_omega).

``params`` is ``(E, nu, sigma0, edot0, n)`` for the elastic-viscoplastic
(Norton) law and ``(E, nu)`` for the linear-elastic law.
"""
import ctypes

import numpy as np

from . import build as _build

KIND_ELASTIC = 0
KIND_NORTON = 1
KIND_MICHEL_SUQUET = 2

# z = P y with y = (z11, z22, g23, g13, g12) and z33 = -z11 - z22 (Sec. 6:
# one component of the deviatoric viscoplastic strain is eliminated).
P_MATRIX = np.array([
    [1, 0, 0, 0, 0],
    [0, 1, 0, 0, 0],
    [-1, -1, 0, 0, 0],
    [0, 0, 1, 0, 0],
    [0, 0, 0, 1, 0],
    [0, 0, 0, 0, 1],
], dtype=np.float64)
_W = np.diag([2 / 3, 2 / 3, 2 / 3, 1 / 3, 1 / 3, 1 / 3])
G_MATRIX = P_MATRIX.T @ _W @ P_MATRIX

_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        lib.ora_update.argtypes = [ctypes.c_int, _dp, ctypes.c_int64, _dp, _dp, ctypes.c_double,
                                   _dp, _dp, _dp, _ip]
        lib.ora_update.restype = ctypes.c_int
        lib.ora_radial_return.argtypes = [_dp, ctypes.c_int64, _dp, _dp, ctypes.c_double, _dp, _dp]
        lib.ora_psi.argtypes = [_dp, _dp, _dp]
        lib.ora_psi.restype = ctypes.c_double
        lib.ora_psi_y.argtypes = [_dp, _dp, _dp, _dp]
        lib.ora_psi_yy.argtypes = [_dp, _dp]
        lib.ora_stress.argtypes = [_dp, _dp, _dp, _dp]
        lib.ora_phi.argtypes = [_dp, _dp]
        lib.ora_phi.restype = ctypes.c_double
        lib.ora_phi_v.argtypes = [_dp, _dp, _dp]
        lib.ora_phi_vv.argtypes = [_dp, _dp, _dp]
        lib.ora_phi_vv.restype = ctypes.c_int
        lib.ora_residual.argtypes = [_dp, _dp, _dp, _dp, ctypes.c_double, _dp]
        lib.ora_newton_matrix.argtypes = [_dp, _dp, _dp, ctypes.c_double, _dp]
        lib.ora_newton_matrix.restype = ctypes.c_int
        lib.ora_Pi.argtypes = [_dp, _dp, _dp, _dp, ctypes.c_double]
        lib.ora_Pi.restype = ctypes.c_double
        lib.ora_max_threads.restype = ctypes.c_int
        lib.ora_newton_matrix_batch.argtypes = [_dp, ctypes.c_int64, _dp, _dp, ctypes.c_double, _dp, _dp]
        lib.ora_update_ode.argtypes = [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int64, _dp, _dp, _dp, _dp,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp, _dp, _dp,
                                       _dp, _ip]
        lib.ora_update_ode.restype = ctypes.c_int
        lib.ora_psi_force_a.argtypes = [_dp, _dp, _dp, _dp]
        lib.ora_psi_force_ms.argtypes = [_dp, _dp, _dp, _dp]
        lib.ora_psi_force_aaa.argtypes = [ctypes.c_int, _dp, _dp, _dp, _dp, _dp]
        lib.ora_psi_force_ms.restype = ctypes.c_double
        lib.ora_gen_stress_ms.argtypes = [_dp, _dp, _dp, _dp]
        lib.ora_flop_pieces.argtypes = [_dp, _dp, _dp, _dp, ctypes.c_double, ctypes.POINTER(ctypes.c_int64)]
        lib.ora_flop_pieces.restype = ctypes.c_int
        _lib = lib
    return _lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return a.ctypes.data_as(_dp)


def _params(params):
    p = list(params) + [0.0] * (5 - len(params))
    if len(params) == 2:
        p[3] = 1.0
        p[4] = 1.0
    return _f64(p)


def max_threads() -> int:
    """Number of OpenMP threads the oracle's voxel loops use."""
    return int(_load().ora_max_threads())


def lame(E, nu):
    """Lame constants (lambda, mu) of an isotropic material."""
    return E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))


def update(kind, params, eps, z_n, h, tangent=False, info=False):
    """Implicit-Euler GSM update of ``n`` independent voxels (Sec. 4.1).

    Returns ``sigma[n,6]``, ``z[n,6]`` and optionally ``C_t[n,6,6]`` (Eq.
    tangent_formula) and ``info[n,3]`` = (line-search iterations, Newton
    iterations, flags with 1=converged, 2=non-finite, 4=cap, 8=not SPD).
    """
    lib = _load()
    eps = _f64(eps, (-1, 6))
    n = eps.shape[0]
    z_n = _f64(z_n, (n, 6))
    sig = np.empty((n, 6))
    z = np.empty((n, 6))
    Ct = np.empty((n, 6, 6)) if tangent else None
    inf = np.empty((n, 3), dtype=np.int32) if info else None
    rc = lib.ora_update(int(kind), _ptr(_params(params)), n, _ptr(eps), _ptr(z_n), float(h),
                        _ptr(sig), _ptr(z), _ptr(Ct) if tangent else None,
                        inf.ctypes.data_as(_ip) if info else None)
    if rc != 0:
        raise ValueError(f"ora_update failed with code {rc}")
    out = [sig, z]
    if tangent:
        out.append(Ct)
    if info:
        out.append(inf)
    return tuple(out)


def radial_return(params, eps, z_n, h):
    """Conventional scalar radial return (Sec. 4, Simo-Hughes) -- an independent pin."""
    lib = _load()
    eps = _f64(eps, (-1, 6))
    n = eps.shape[0]
    z_n = _f64(z_n, (n, 6))
    sig = np.empty((n, 6))
    z = np.empty((n, 6))
    lib.ora_radial_return(_ptr(_params(params)), n, _ptr(eps), _ptr(z_n), float(h), _ptr(sig), _ptr(z))
    return sig, z


def psi(params, eps, y):
    return _load().ora_psi(_ptr(_params(params)), _ptr(_f64(eps)), _ptr(_f64(y)))


def psi_y(params, eps, y):
    g = np.empty(5)
    _load().ora_psi_y(_ptr(_params(params)), _ptr(_f64(eps)), _ptr(_f64(y)), _ptr(g))
    return g


def psi_yy(params):
    H = np.empty((5, 5))
    _load().ora_psi_yy(_ptr(_params(params)), _ptr(H))
    return H


def stress(params, eps, y):
    s = np.empty(6)
    _load().ora_stress(_ptr(_params(params)), _ptr(_f64(eps)), _ptr(_f64(y)), _ptr(s))
    return s


def phi(params, v):
    return _load().ora_phi(_ptr(_params(params)), _ptr(_f64(v)))


def phi_v(params, v):
    g = np.empty(5)
    _load().ora_phi_v(_ptr(_params(params)), _ptr(_f64(v)), _ptr(g))
    return g


def phi_vv(params, v):
    H = np.empty((5, 5))
    rc = _load().ora_phi_vv(_ptr(_params(params)), _ptr(_f64(v)), _ptr(H))
    return H if rc == 0 else None


def residual(params, eps, y, y_n, h):
    R = np.empty(5)
    _load().ora_residual(_ptr(_params(params)), _ptr(_f64(eps)), _ptr(_f64(y)), _ptr(_f64(y_n)),
                         float(h), _ptr(R))
    return R


def newton_matrix(params, y, y_n, h):
    K = np.empty((5, 5))
    rc = _load().ora_newton_matrix(_ptr(_params(params)), _ptr(_f64(y)), _ptr(_f64(y_n)), float(h), _ptr(K))
    return K if rc == 0 else None


def incremental_potential(params, eps, y, y_n, h):
    """Pi(y) = psi(eps, y) + h phi((y - y_n)/h)."""
    return _load().ora_Pi(_ptr(_params(params)), _ptr(_f64(eps)), _ptr(_f64(y)), _ptr(_f64(y_n)), float(h))




def newton_matrix_batch(params, y, y_n, h):
    """K = psi_yy + phi_vv/h and phi_vv at n states; y, y_n [n, 5] -> ([n,5,5], [n,5,5])."""
    y = _f64(y, (-1, 5))
    n = y.shape[0]
    y_n = _f64(y_n, (n, 5))
    K = np.empty((n, 5, 5))
    H = np.empty((n, 5, 5))
    _load().ora_newton_matrix_batch(_ptr(_params(params)), n, _ptr(y), _ptr(y_n), float(h), _ptr(K), _ptr(H))
    return K, H


ODE_METHODS = {"ode23": 0, "ode12": 1, "ode23s": 2}


def update_ode23(params, eps_n, eps, z_n, h, rtol=1e-3, atol=1e-6, max_steps=100000, tangent=False, info=False,
                 kind=KIND_NORTON, alpha_n=None, method="ode23"):
    """Material update by ode23 (Sec. 4.3, stress-driven error control Sec. 4.5),
    or by ode12 (explicit Euler / Heun pair, same control) with method="ode12",
    or by ode23s (Shampine-Reichelt Rosenbrock triple) with method="ode23s".

    kind KIND_NORTON: params (E, nu, sigma0, edot0, n); KIND_MICHEL_SUQUET:
    params (E, nu, sigma_Y, H, edot0, sigma_d, n) with the equivalent plastic
    strain alpha as a further internal variable (alpha_n: (n,) or None = 0).
    eps_n, eps, z_n: (n, 6); returns sigma, z [, alpha (Michel-Suquet)]
    [, tangent (n, 6, 6)] [, info (n, 3) = accepted substeps, rejected
    substeps, flags]."""
    lib = _load()
    eps_n = _f64(eps_n).reshape(-1, 6)
    eps = _f64(eps).reshape(-1, 6)
    z_n = _f64(z_n).reshape(-1, 6)
    n = eps.shape[0]
    sig = np.zeros((n, 6))
    z = np.zeros((n, 6))
    alpha = np.zeros(n)
    a_n = _f64(alpha_n).reshape(n) if alpha_n is not None else None
    C = np.zeros((n, 6, 6)) if tangent else None
    inf = np.zeros((n, 3), dtype=np.int32)
    prm = _f64(list(params) + [0.0] * (7 - len(params)))
    rc = lib.ora_update_ode(int(kind), ODE_METHODS[method], _ptr(prm), ctypes.c_int64(n), _ptr(eps_n), _ptr(eps),
                            _ptr(z_n), _ptr(a_n) if a_n is not None else None, ctypes.c_double(h),
                            ctypes.c_double(rtol), ctypes.c_double(atol), ctypes.c_int(max_steps), _ptr(sig), _ptr(z),
                            _ptr(alpha), _ptr(C) if tangent else None,
                            inf.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    if rc != 0:
        raise ValueError("update_ode23: unsupported law kind")
    out = [sig, z]
    if kind == KIND_MICHEL_SUQUET:
        out.append(alpha)
    if tangent:
        out.append(C)
    if info:
        out.append(inf)
    return tuple(out)


def psi_force_ms(params, A):
    """(Psi, Psi_A, Psi_AA) of the Michel-Suquet force potential at A = (A_y, A_alpha) (6,)."""
    lib = _load()
    A = _f64(A).reshape(6)
    g = np.zeros(6)
    H = np.zeros((6, 6))
    v = lib.ora_psi_force_ms(_ptr(_f64(params)), _ptr(A), _ptr(g), _ptr(H))
    return v, g, H


def gen_stress_ms(params, eps, y6):
    """Generalized stress A = -d omega/d(y, alpha) of the Michel-Suquet law (6,)."""
    lib = _load()
    A = np.zeros(6)
    lib.ora_gen_stress_ms(_ptr(_f64(params)), _ptr(_f64(eps).reshape(6)), _ptr(_f64(y6).reshape(6)), _ptr(A))
    return A


def psi_force_a(params, A):
    """(Psi_A, Psi_AA) of the Norton force potential at A (5,)."""
    lib = _load()
    A = _f64(A).reshape(5)
    g = np.zeros(5)
    H = np.zeros((5, 5))
    lib.ora_psi_force_a(_ptr(_params(params)), _ptr(A), _ptr(g), _ptr(H))
    return g, H


def psi_force_aaa(params, A, u, v, kind=KIND_NORTON):
    """Psi_AAA[u, v] of the force potential (Norton: 5 entries; Michel-Suquet: 6)."""
    lib = _load()
    k = 5 if kind == KIND_NORTON else 6
    out = np.zeros(k)
    prm = _f64(list(params) + [0.0] * (7 - len(params)))
    lib.ora_psi_force_aaa(int(kind), _ptr(prm), _ptr(_f64(A).reshape(k)), _ptr(_f64(u).reshape(k)),
                          _ptr(_f64(v).reshape(k)), _ptr(out))
    return out


FLOP_PIECES = ("predictor", "line", "newton", "residual", "subst", "stress", "tangent")
FLOP_KINDS = ("add", "mul", "div", "sqrt", "pow")


def flop_pieces(params, eps, z_n, y, h):
    """Algorithmic flops of the pieces of the implicit-Euler update (Sec. 4.1)
    of the Norton law, counted on the oracle's own statements at a flowing
    state (``y`` the converged 5 unknowns, y != y_n).  Returns
    {piece: {kind: count}} for the pieces of ``FLOP_PIECES`` and the kinds
    of ``FLOP_KINDS`` (add/sub, mul, div, sqrt: one flop each; pow apart)."""
    out = np.zeros((len(FLOP_PIECES), len(FLOP_KINDS)), dtype=np.int64)
    rc = _load().ora_flop_pieces(_ptr(_params(params)), _ptr(_f64(eps)), _ptr(_f64(z_n)), _ptr(_f64(y)), float(h),
                                 out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    if rc != 0:
        raise ValueError("flop_pieces needs a flowing state (y != y_n)")
    return {p: dict(zip(FLOP_KINDS, map(int, row))) for p, row in zip(FLOP_PIECES, out)}
