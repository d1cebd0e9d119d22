"""Moulinec-Suquet basic scheme in plain numpy, FP64 -- TEST INFRASTRUCTURE ONLY.

The paper drives the material law by the FFT-based basic scheme of Moulinec
and Suquet (Sec. 1; Sec. 3 "Material Law Evaluations": a reference stiffness
C^ref, fixed or updated per step, and one material evaluation without tangent
per iteration and voxel).  The paper cites the scheme without restating its
formulas; this module writes out the standard scheme:

  * periodic cell [0,1)^3 on an N^3 voxel grid, frequencies xi = 2 pi k,
    k in {0..ceil(N/2)-1, -floor(N/2)..-1} per axis;
  * isotropic reference medium (lambda0, mu0) = midpoints of the phases'
    elastic Lame constants (fixed C^ref, Sec. 3);
  * Green operator applied to a symmetric tau with q = tau xi:
      (Gamma0 : tau)_kh = (xi_h q_k + xi_k q_h) / (2 mu0 |xi|^2)
                          - (lambda0 + mu0) / (mu0 (lambda0 + 2 mu0)) (xi.q) xi_k xi_h / |xi|^4
  * iteration  eps^(i+1)^(xi) = eps^i^(xi) - Gamma0(xi) : sigma^i^(xi)  (xi != 0),
               eps^(i+1)^(0)  = N^3 E_k;
  * equilibrium error e = sqrt(sum_xi |xi . c(xi)|^2) / |<sigma>|_F with
    c = sigma^ / N^3 (|.|_F the tensor Frobenius norm);
  * load step k: eps <- eps + (E_k - E_{k-1}) uniformly, iterate until
    e < tol, then z_n <- z and Sigma_k = <sigma>.

Even-N convention (a reading; the paper is silent): a mode whose index
vector contains the Nyquist index N/2 together with any other nonzero index
has no Hermitian-consistent Green operator (xi_i xi_j flips sign between the
two aliases); there Gamma0 := 0 and the mode is excluded from the error sum.
Pure-axis Nyquist modes (N/2, 0, 0) etc. keep the exact operator.

Strain-like Voigt vectors carry engineering shears, so the strain update of a
shear component is 2 (Gamma0 : tau)_ij.
"""
import numpy as np

from . import material as M

VOIGT = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]


def reference_medium(laws):
    """(lambda0, mu0): midpoints over the phases' elastic Lame constants."""
    lm = [M.lame(p[1][0], p[1][1]) for p in laws]
    lams = [a for a, _ in lm]
    mus = [b for _, b in lm]
    return 0.5 * (min(lams) + max(lams)), 0.5 * (min(mus) + max(mus))


def wavevectors(N):
    """Integer frequency vectors k (3, N, N, N) and the mask of excluded modes."""
    k1 = np.fft.fftfreq(N, d=1.0 / N).round().astype(np.int64)
    kx, ky, kz = np.meshgrid(k1, k1, k1, indexing="ij")
    k = np.stack([kx, ky, kz]).astype(np.float64)
    excluded = np.zeros((N, N, N), dtype=bool)
    if N % 2 == 0:
        nyq = [np.abs(c) == N // 2 for c in (kx, ky, kz)]
        nonzero = [c != 0 for c in (kx, ky, kz)]
        n_nonzero = nonzero[0].astype(int) + nonzero[1] + nonzero[2]
        any_nyq = nyq[0] | nyq[1] | nyq[2]
        excluded = any_nyq & (n_nonzero >= 2)
    return k, excluded


def voigt_to_tensor_field(a, engineering):
    """(..., 6) Voigt -> (3, 3, ...) symmetric tensor field."""
    f = 0.5 if engineering else 1.0
    T = np.empty((3, 3) + a.shape[:-1], dtype=a.dtype)
    for c, (i, j) in enumerate(VOIGT):
        s = a[..., c] * (f if i != j else 1.0)
        T[i, j] = s
        T[j, i] = s
    return T


def gamma0_apply(tau_hat, lam0, mu0, N):
    """Gamma0 : tau for every mode; tau_hat (3, 3, N, N, N) complex.

    Returns the strain-like Voigt field (N, N, N, 6) with engineering shears;
    the zero mode and the excluded Nyquist modes are set to 0.
    """
    k, excluded = wavevectors(N)
    xi = 2.0 * np.pi * k
    xi2 = (xi ** 2).sum(axis=0)
    xi2_safe = np.where(xi2 == 0, 1.0, xi2)
    q = np.einsum("ij...,j...->i...", tau_hat, xi)
    xq = np.einsum("i...,i...->...", xi, q)
    a = 1.0 / (2.0 * mu0 * xi2_safe)
    b = (lam0 + mu0) / (mu0 * (lam0 + 2.0 * mu0)) / xi2_safe ** 2
    out = np.empty((N, N, N, 6), dtype=np.complex128)
    for c, (i, j) in enumerate(VOIGT):
        d = a * (xi[j] * q[i] + xi[i] * q[j]) - b * xq * xi[i] * xi[j]
        out[..., c] = d if i == j else 2.0 * d
    kill = (xi2 == 0) | excluded
    out[kill] = 0.0
    return out


def equilibrium_error(sig_hat, mean_sig, N, floor):
    """e = sqrt(sum |xi . c|^2) / max(|<sigma>|_F, floor), c = sigma^/N^3."""
    k, excluded = wavevectors(N)
    xi = 2.0 * np.pi * k
    T = voigt_to_tensor_field(np.moveaxis(sig_hat, 0, -1), engineering=False) / N ** 3
    q = np.einsum("ij...,j...->i...", T, xi)
    w = (np.abs(q) ** 2).sum(axis=0)
    w[excluded] = 0.0
    num = np.sqrt(w.sum())
    Sm = voigt_to_tensor_field(np.asarray(mean_sig), engineering=False)
    den = max(np.sqrt((Sm ** 2).sum()), floor)
    return num / den


def material(eps, z_n, phase, laws, h, tangent=False, eps_n=None, ode=None, ode_method="ode23"):
    """One material evaluation of every voxel: laws[p] = (kind, params) for phase p.

    Implicit Euler (Sec. 4.1) unless ``ode`` = (rtol, atol): then the ode23
    (or, with ode_method="ode12", the Euler/Heun) update of the force-potential
    form over the step (Sec. 4.3) from the strain eps_n of the previous step;
    z_n has 7 columns there (z, alpha)."""
    n = eps.shape[0]
    nz = z_n.shape[1]
    sig = np.empty((n, 6))
    z = np.empty((n, nz))
    Ct = np.empty((n, 6, 6)) if tangent else None
    for p, (kind, params) in enumerate(laws):
        idx = np.nonzero(phase == p)[0]
        if idx.size == 0:
            continue
        if ode is None or kind == M.KIND_ELASTIC:
            if kind == M.KIND_MICHEL_SUQUET:
                raise ValueError("the Michel-Suquet law needs the ode23 update")
            out = M.update(kind, params, eps[idx], z_n[idx, :6], h, tangent=tangent)
            sig[idx] = out[0]
            z[idx, :6] = out[1]
            if nz > 6:
                z[idx, 6:] = z_n[idx, 6:]
            if tangent:
                Ct[idx] = out[2]
        else:
            kw = {"alpha_n": z_n[idx, 6]} if kind == M.KIND_MICHEL_SUQUET else {}
            out = M.update_ode23(params, eps_n[idx], eps[idx], z_n[idx, :6], h, rtol=ode[0], atol=ode[1],
                                 tangent=tangent, kind=kind, method=ode_method, **kw)
            sig[idx] = out[0]
            z[idx, :6] = out[1]
            k = 2
            if kind == M.KIND_MICHEL_SUQUET:
                z[idx, 6] = out[2]
                k = 3
            elif nz > 6:
                z[idx, 6:] = z_n[idx, 6:]
            if tangent:
                Ct[idx] = out[k]
    return (sig, z, Ct) if tangent else (sig, z)


def isotropic_measures(Ct):
    """Per-voxel isotropic measures of tangents Ct (n, 6, 6) (stress-like rows,
    engineering-shear columns): 3k = J::C = (1/3) sum_{i,j<3} C_ij and
    10 mu = tr_Mandel(C) - 3k, tr_Mandel = C11 + C22 + C33 + 2 (C44 + C55 + C66).
    For an isotropic C they are its bulk and shear moduli."""
    three_k = Ct[:, :3, :3].sum(axis=(1, 2)) / 3.0
    tr = Ct[:, 0, 0] + Ct[:, 1, 1] + Ct[:, 2, 2] + 2.0 * (Ct[:, 3, 3] + Ct[:, 4, 4] + Ct[:, 5, 5])
    return three_k / 3.0, (tr - three_k) / 10.0


def reference_from_tangents(Ct):
    """Per-step reference medium (Sec. 3: adjusted to the current tangential
    stiffness): k0, mu0 the midpoints of the per-voxel bulk and shear measures,
    lambda0 = k0 - 2 mu0 / 3.  For isotropic elastic phases this is the fixed
    reference of reference_medium."""
    k, mu = isotropic_measures(Ct)
    k0 = 0.5 * (k.min() + k.max())
    mu0 = 0.5 * (mu.min() + mu.max())
    return k0 - 2.0 * mu0 / 3.0, mu0


def reference_stiffness(lam0, mu0):
    """Isotropic C0 (Voigt, engineering shears)."""
    C = np.zeros((6, 6))
    C[:3, :3] = lam0
    C[:3, :3] += 2.0 * mu0 * np.eye(3)
    C[3:, 3:] = mu0 * np.eye(3)
    return C


def solve(phase, laws, loads, hs, tol=1e-8, max_iter=10000, forced_iters=None,
          eps0=None, zn0=None, E_prev0=None, record=False, stress_mask=None, Sigma_target=None,
          ref_update=False, ode=None, ode_method="ode23"):
    """Load-history solve of the basic scheme.

    phase : (N, N, N) uint8 phase ids, voxel (i, j, k) with k fastest.
    laws  : list of (kind, params) per phase id.
    loads : (n_steps, 6) macroscopic strains E_k (engineering shears).
    hs    : step sizes h_k.
    forced_iters : optional per-step number of material evaluations to run
                   regardless of tol (used for iteration-matched parity).
    stress_mask  : optional 6 booleans: components whose macroscopic STRESS is
                   prescribed (mixed boundary conditions; the others prescribe the
                   strain E_k).  Their mean strain is an unknown, corrected after
                   each evaluation by dE_s = (C0_ss)^-1 (Sigma_s - <sigma>_s), and
                   the stopping error is max(e, |Sigma_s - <sigma>_s|_F / |<sigma>|_F).
    Sigma_target : (n_steps, 6) prescribed stresses (default 0).
    ref_update   : adjust the reference medium at the start of every load step
                   to the tangents of a material evaluation at the predicted
                   strain (Sec. 3), instead of the fixed elastic reference.
    ode          : None (implicit Euler) or (rtol, atol): the laws integrate the
                   force-potential form over each step by ode23 from the strain
                   of the previous step (Sec. 4.3); the internal variables then
                   have 7 columns (z, alpha) when a phase is a Michel-Suquet law.
    ode_method   : "ode23", "ode12" (explicit Euler / Heun pair) or "ode23s"
                   (Shampine-Reichelt Rosenbrock triple).

    Returns dict with Sigma (n_steps, 6), iters (n_steps,), errors (list per
    step), eps and z (N^3, 6) at the end, and the per-step (eps, z) history if
    ``record``.
    """
    phase = np.asarray(phase)
    N = phase.shape[0]
    nvox = N ** 3
    ph = phase.reshape(-1)
    lam0, mu0 = reference_medium(laws)
    loads = np.asarray(loads, dtype=np.float64).reshape(-1, 6)
    eps = np.zeros((nvox, 6)) if eps0 is None else np.array(eps0, dtype=np.float64).reshape(nvox, 6)
    nz = 7 if any(k == M.KIND_MICHEL_SUQUET for k, _ in laws) else 6
    z_n = np.zeros((nvox, nz)) if zn0 is None else np.array(zn0, dtype=np.float64).reshape(nvox, nz)
    eps_prev = None
    E_prev = np.zeros(6) if E_prev0 is None else np.asarray(E_prev0, dtype=np.float64)
    mask = np.zeros(6, dtype=bool) if stress_mask is None else np.asarray(stress_mask, dtype=bool)
    S_t = np.zeros((loads.shape[0], 6)) if Sigma_target is None else np.asarray(Sigma_target, float).reshape(-1, 6)
    wF = np.array([1.0, 1.0, 1.0, 2.0, 2.0, 2.0])  # tensor Frobenius weights of stress-like Voigt vectors
    E_mean = E_prev.copy()                          # the current macroscopic strain
    Sigma, iters, errors, hist, Es, refs = [], [], [], [], [], []
    for step, (E_k, h) in enumerate(zip(loads, hs)):
        eps_prev = eps.copy()  # the strain at t_n of every voxel (the ode23 update integrates from it)
        E_start = np.where(mask, E_mean, E_k)
        eps = eps + (E_start - E_mean)[None, :]
        E_mean = E_start.copy()
        if ref_update:
            _, _, Ct = material(eps, z_n, ph, laws, h, tangent=True, eps_n=eps_prev, ode=ode, ode_method=ode_method)
            lam0, mu0 = reference_from_tangents(Ct)
        refs.append((lam0, mu0))
        floor = mu0 * 1e-6
        C0 = reference_stiffness(lam0, mu0)
        C0ss_inv = np.linalg.inv(C0[np.ix_(mask, mask)]) if mask.any() else None
        errs = []
        n_eval = 0
        while True:
            sig, z = material(eps, z_n, ph, laws, h, eps_n=eps_prev, ode=ode, ode_method=ode_method)
            n_eval += 1
            sig_hat = np.stack([np.fft.fftn(sig[:, c].reshape(N, N, N)) for c in range(6)])
            mean_sig = sig.mean(axis=0)
            e = equilibrium_error(sig_hat, mean_sig, N, floor)
            if mask.any():
                r = (S_t[step] - mean_sig)[mask]
                den = max(np.sqrt(np.sum(wF * mean_sig ** 2)), floor)
                e = max(e, np.sqrt(np.sum(wF[mask] * r ** 2)) / den)
            errs.append(e)
            if forced_iters is not None:
                if n_eval >= forced_iters[step]:
                    break
            elif e < tol or n_eval >= max_iter:
                break
            if mask.any():
                E_mean[mask] = E_mean[mask] + C0ss_inv @ r
            tau = voigt_to_tensor_field(np.moveaxis(sig_hat, 0, -1), engineering=False)
            d_hat = gamma0_apply(tau, lam0, mu0, N)
            eps_hat = np.stack([np.fft.fftn(eps[:, c].reshape(N, N, N)) for c in range(6)], axis=-1)
            eps_hat = eps_hat - d_hat
            eps_hat[0, 0, 0, :] = nvox * E_mean
            eps = np.stack([np.fft.ifftn(eps_hat[..., c]).real.reshape(-1) for c in range(6)], axis=-1)
        z_n = z
        Sigma.append(mean_sig)
        Es.append(E_mean.copy())
        iters.append(n_eval)
        errors.append(errs)
        if record:
            hist.append((eps.copy(), z_n.copy(), sig.copy()))
    out = {"Sigma": np.array(Sigma), "iters": np.array(iters), "errors": errors,
           "eps": eps, "z": z_n, "sigma": sig, "lam0": lam0, "mu0": mu0, "E": np.array(Es),
           "reference": np.array(refs)}
    if record:
        out["history"] = hist
    return out


# ------------------------------------------------------------------ adjoint
# Gradient of J = w . Sigma_K (final mean stress) with respect to the
# parameters theta = (E, sigma0, n) of one Norton phase, through the whole
# load history (the paper's AD is local to a voxel, Sec. 5; this is the
# discrete adjoint of the implicit-Euler update plus the basic scheme).
#
# Step k maps (z_{k-1}, theta) to (sigma_k, z_k) through the equilibrium
# constraint P_V sigma(E_k + u) = 0 on compatible zero-mean fluctuations u.
# Given adjoints (g_sig, g_z) of (sigma_k, z_k):
#   a_u   = C_t^T g_sig + (dz/deps)^T g_z,          dz/deps = P K^-1 P^T C
#   find compatible zero-mean lam with P_V (C_t lam) = P_V a_u
#   a     = g_sig - lam
#   b     = K^-1 (P^T g_z - P^T C a)
#   g_{z,k-1} = (phi_vv / h) b   on the components (11, 22, 23, 13, 12)
#   dJ/dtheta += sum_x a . d sigma/d theta|_y - b . dR/d theta
# with R = psi_y + phi_v and, at the converged state, phi_v = P^T sigma:
#   d sigma/dE|_y = sigma/E, dR/dE = -P^T sigma/E,
#   dR/d sigma0 = P^T sigma / sigma0,
#   dR/dn = P^T sigma * (-ln(s/edot0) / n^2),  s = sqrt(v^T G v), v = (y - y_n)/h.
# Voxels without flow (y = y_n exactly) have dy/dy_n = I: g_{z,k-1} = P^T g_z - P^T C a.

Y_IDX = [0, 1, 3, 4, 5]


def stiffness_voigt(E, nu):
    lam, mu = M.lame(E, nu)
    C = np.zeros((6, 6))
    C[:3, :3] = lam
    C[:3, :3] += 2 * mu * np.eye(3)
    C[3:, 3:] = mu * np.eye(3)
    return C


def solve_taped(phase, laws, loads, hs, tol=1e-12, max_iter=100000):
    """Forward solve keeping per-step checkpoints (eps_k, z_{k-1})."""
    r = solve(phase, laws, loads, hs, tol=tol, max_iter=max_iter, record=True)
    nvox = np.asarray(phase).size
    tape = []
    z_prev = np.zeros((nvox, 6))
    for eps_k, z_k, _ in r["history"]:
        tape.append((eps_k, z_prev))
        z_prev = z_k
    r["tape"] = tape
    return r


def _lambda_solve(Ct, a_u, N, lam0, mu0, tol, max_iter):
    """Compatible zero-mean lam with P_V(C_t lam) = P_V(a_u) by the basic-scheme fixed point."""
    nvox = N ** 3
    lam = np.zeros((nvox, 6))
    first = None
    for it in range(max_iter):
        tau = np.einsum("nij,nj->ni", Ct, lam) - a_u
        tau_hat = np.stack([np.fft.fftn(tau[:, c].reshape(N, N, N)) for c in range(6)])
        k, excluded = wavevectors(N)
        xi = 2 * np.pi * k
        T = voigt_to_tensor_field(np.moveaxis(tau_hat, 0, -1), engineering=False)
        q = np.einsum("ij...,j...->i...", T, xi)
        wq = (np.abs(q) ** 2).sum(axis=0)
        wq[excluded] = 0.0
        err = np.sqrt(wq.sum())
        first = err if first is None else first
        if err <= tol * max(first, 1e-300):
            break
        d_hat = gamma0_apply(voigt_to_tensor_field(np.moveaxis(tau_hat, 0, -1), engineering=False), lam0, mu0, N)
        lam_hat = np.stack([np.fft.fftn(lam[:, c].reshape(N, N, N)) for c in range(6)], axis=-1) - d_hat
        lam_hat[0, 0, 0, :] = 0.0
        lam = np.stack([np.fft.ifftn(lam_hat[..., c]).real.reshape(-1) for c in range(6)], axis=-1)
    return lam, it + 1


def adjoint(phase, laws, loads, hs, tape, w, phase_id, tol=1e-12, max_iter=100000):
    """dJ/d(E, sigma0, n) of phase `phase_id` for J = w . Sigma_K."""
    ph = np.asarray(phase).reshape(-1)
    N = np.asarray(phase).shape[0]
    nvox = N ** 3
    lam0, mu0 = reference_medium(laws)
    kind, prm = laws[phase_id]
    assert kind == M.KIND_NORTON
    E_mod, nu, sigma0, edot0, n_exp = prm
    Pm = M.P_MATRIX
    Gm = M.G_MATRIX
    w = np.asarray(w, dtype=np.float64)
    K_steps = len(tape)
    g_z = np.zeros((nvox, 6))
    grad = np.zeros(3)
    lam_iters = []
    for k in range(K_steps - 1, -1, -1):
        eps_k, z_prev = tape[k]
        h = hs[k]
        g_sig = np.tile(w / nvox, (nvox, 1)) if k == K_steps - 1 else np.zeros((nvox, 6))
        Ct = np.zeros((nvox, 6, 6))
        a_u = np.zeros((nvox, 6))
        local = {}
        for p, (kind_p, prm_p) in enumerate(laws):
            idx = np.nonzero(ph == p)[0]
            if idx.size == 0:
                continue
            sig, z, Ct_p = M.update(kind_p, prm_p, eps_k[idx], z_prev[idx], h, tangent=True)
            Ct[idx] = Ct_p
            if kind_p == M.KIND_NORTON:
                y, yn = z[:, Y_IDX], z_prev[idx][:, Y_IDX]
                Kmat, Hphi = M.newton_matrix_batch(prm_p, y, yn, h)
                C = stiffness_voigt(prm_p[0], prm_p[1])
                gy = g_z[idx] @ Pm                           # P^T g_z
                t = np.linalg.solve(Kmat, gy[..., None])[..., 0]
                a_u[idx] = np.einsum("nji,nj->ni", Ct_p, g_sig[idx]) + (t @ Pm.T) @ C.T  # C_t^T g + C P t
                local[p] = (idx, sig, y, yn, Kmat, Hphi, C)
            else:
                a_u[idx] = np.einsum("nji,nj->ni", Ct_p, g_sig[idx])
        lam, it = _lambda_solve(Ct, a_u, N, lam0, mu0, tol, max_iter)
        lam_iters.append(it)
        a = g_sig - lam
        g_z_prev = np.zeros((nvox, 6))
        for p, (idx, sig, y, yn, Kmat, Hphi, C) in local.items():
            rhs = g_z[idx] @ Pm - (a[idx] @ C.T) @ Pm      # P^T g_z - P^T C a
            b = np.linalg.solve(Kmat, rhs[..., None])[..., 0]
            flow = np.any(y != yn, axis=1)
            g_yn = np.where(flow[:, None], np.einsum("nij,nj->ni", Hphi, b) / h, rhs)
            g_z_prev[idx[:, None], np.array(Y_IDX)[None, :]] = g_yn
            if p != phase_id:
                continue
            Pts = sig @ Pm                                   # P^T sigma
            v = (y - yn) / h
            s = np.sqrt(np.einsum("ni,ij,nj->n", v, Gm, v))
            logt = np.where(s > 0, np.log(np.where(s > 0, s, 1.0) / edot0), 0.0)
            grad[0] += np.sum(a[idx] * sig) / E_mod + np.sum(b * Pts) / E_mod
            grad[1] += -np.sum(b * Pts) / sigma0
            grad[2] += np.sum(np.sum(b * Pts, axis=1) * logt) / n_exp ** 2
        g_z = g_z_prev
    return grad, lam_iters
