"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This package holds input recipes only -- random draws, microstructure
geometry and load histories -- and none of the material-law or basic-scheme
arithmetic.  It imports neither the CUDA package nor the oracle.

Recipes (the paper's workload -- a 150^3 GeoDict short-fibre metal-matrix
composite, Sec. 3 -- is not available; these stand in for it):

* ``material_batch``: independent voxels, eps ~ U[-a, a]^6 on the Voigt vector
  (engineering shears), deviatoric z_n with (z11, z22, g23, g13, g12) ~
  U[-b, b]^5 i.i.d. and z33 = -z11 - z22.
* ``sphere_phase``: one centred spherical inclusion; a voxel (i, j, k) is
  inside when its centre (i+1/2, j+1/2, k+1/2) lies within r of (N/2,N/2,N/2),
  r = (3 f N^3 / (4 pi))^(1/3).
* ``rsa_cylinders``: random sequential adsorption of straight cylinders with
  axes in the x-y plane, uniform centres, angle U[0, pi), periodic images;
  a candidate is accepted when its axis keeps a distance >= 2r + 1 from every
  accepted axis; stops at the target volume fraction.
* ``rsa_spheres``: the same for spheres of radius r (distance >= 2r + 1).
* ``laminate_phase``: two layers normal to x.
* load histories: ``ramp`` (E_k = (k/n) * E_final).
"""
import math

import numpy as np


def material_batch(n, seed=0, eps_amp=0.02, z_amp=0.005):
    """(eps[n,6], z_n[n,6]) float64, AoS."""
    rng = np.random.Generator(np.random.PCG64(seed))
    eps = rng.uniform(-eps_amp, eps_amp, size=(n, 6))
    y = rng.uniform(-z_amp, z_amp, size=(n, 5))
    zn = np.empty((n, 6))
    zn[:, 0] = y[:, 0]
    zn[:, 1] = y[:, 1]
    zn[:, 2] = -y[:, 0] - y[:, 1]
    zn[:, 3:] = y[:, 2:]
    return eps, zn


def sphere_radius(N, frac):
    return (3.0 * frac * N ** 3 / (4.0 * math.pi)) ** (1.0 / 3.0)


def sphere_phase(N, frac):
    """uint8 (N,N,N): 1 inside the centred sphere, 0 elsewhere."""
    r = sphere_radius(N, frac)
    c = np.arange(N) + 0.5 - N / 2.0
    X, Y, Z = np.meshgrid(c, c, c, indexing="ij")
    return ((X * X + Y * Y + Z * Z) <= r * r).astype(np.uint8)


def laminate_phase(N, n_first):
    """uint8 (N,N,N): phase 1 for x-index < n_first, else 0."""
    ph = np.zeros((N, N, N), dtype=np.uint8)
    ph[:n_first] = 1
    return ph


def _periodic_delta(d, N):
    return d - N * np.round(d / N)


def _seg_point_dist2(p, a, b):
    ab = b - a
    t = np.clip(np.dot(p - a, ab) / max(np.dot(ab, ab), 1e-300), 0.0, 1.0)
    d = p - (a + t * ab)
    return float(np.dot(d, d))


def _segments_intersect_2d(a, b, c, d):
    def orient(p, q, r):
        return (q[0] - p[0]) * (r[1] - p[1]) - (q[1] - p[1]) * (r[0] - p[0])
    o1, o2 = orient(a, b, c), orient(a, b, d)
    o3, o4 = orient(c, d, a), orient(c, d, b)
    return (o1 * o2 < 0) and (o3 * o4 < 0)


def _seg_seg_dist_2d(a, b, c, d):
    if _segments_intersect_2d(a, b, c, d):
        return 0.0
    return math.sqrt(min(_seg_point_dist2(a, c, d), _seg_point_dist2(b, c, d),
                         _seg_point_dist2(c, a, b), _seg_point_dist2(d, a, b)))


def _rasterize_cylinder(ph, centre, theta, radius, length):
    N = ph.shape[0]
    u = np.array([math.cos(theta), math.sin(theta)])
    half = 0.5 * length
    ext_x = abs(u[0]) * half + radius + 1
    ext_y = abs(u[1]) * half + radius + 1
    xs = np.arange(int(math.floor(centre[0] - ext_x)), int(math.ceil(centre[0] + ext_x)) + 1)
    ys = np.arange(int(math.floor(centre[1] - ext_y)), int(math.ceil(centre[1] + ext_y)) + 1)
    zs = np.arange(int(math.floor(centre[2] - radius - 1)), int(math.ceil(centre[2] + radius + 1)) + 1)
    X, Y, Z = np.meshgrid(xs + 0.5, ys + 0.5, zs + 0.5, indexing="ij")
    dx, dy, dz = X - centre[0], Y - centre[1], Z - centre[2]
    t = np.clip(dx * u[0] + dy * u[1], -half, half)
    px, py = dx - t * u[0], dy - t * u[1]
    inside = px * px + py * py + dz * dz <= radius * radius
    I, J, K = np.nonzero(inside)
    flat = np.unique(np.ravel_multi_index((xs[I] % N, ys[J] % N, zs[K] % N), ph.shape))
    new = int(np.count_nonzero(ph.flat[flat] == 0))
    ph.flat[flat] = 1
    return new


def _pt_seg_d2(p, a, b):
    """Squared distance of points p to segments [a, b] (broadcast over leading axes)."""
    ab = b - a
    den = np.maximum(np.sum(ab * ab, axis=-1), 1e-300)
    t = np.clip(np.sum((p - a) * ab, axis=-1) / den, 0.0, 1.0)
    d = p - (a + t[..., None] * ab)
    return np.sum(d * d, axis=-1)


def _seg_seg_dist_2d_many(a, b, C, D):
    """Distances of one 2-D segment [a, b] to many segments [C_i, D_i]."""
    def orient(p, q, r):
        return (q[..., 0] - p[..., 0]) * (r[..., 1] - p[..., 1]) - (q[..., 1] - p[..., 1]) * (r[..., 0] - p[..., 0])
    o1, o2 = orient(a, b, C), orient(a, b, D)
    o3, o4 = orient(C, D, a), orient(C, D, b)
    cross = (o1 * o2 < 0) & (o3 * o4 < 0)
    d2 = np.minimum.reduce([_pt_seg_d2(a, C, D), _pt_seg_d2(b, C, D), _pt_seg_d2(C, a, b), _pt_seg_d2(D, a, b)])
    return np.where(cross, 0.0, np.sqrt(d2))


def rsa_cylinders(N, radius, frac, length, seed=0, max_tries=200000):
    """Periodic RSA of x-y-plane cylinders; returns (uint8 phase, achieved fraction, n_fibres)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ph = np.zeros((N, N, N), dtype=np.uint8)
    A = np.zeros((0, 2))
    B = np.zeros((0, 2))
    Zc = np.zeros(0)
    target = frac * N ** 3
    half = 0.5 * length
    shifts = np.array([(sx, sy) for sx in (-N, 0, N) for sy in (-N, 0, N)], dtype=np.float64)
    tries = 0
    n_acc = 0
    filled = 0
    while filled < target and tries < max_tries:
        tries += 1
        c = rng.uniform(0, N, size=3)
        th = rng.uniform(0, math.pi)
        u = np.array([math.cos(th), math.sin(th)])
        a, b = c[:2] - half * u, c[:2] + half * u
        if n_acc:
            dz = np.abs(_periodic_delta(c[2] - Zc, N))
            near = dz < 2 * radius + 1
            if near.any():
                Cs = A[near][None, :, :] + shifts[:, None, :]
                Ds = B[near][None, :, :] + shifts[:, None, :]
                d2d = _seg_seg_dist_2d_many(a, b, Cs, Ds)
                d3 = np.sqrt(d2d ** 2 + dz[near][None, :] ** 2)
                if np.any(d3 < 2 * radius + 1):
                    continue
        A = np.vstack([A, a[None]])
        B = np.vstack([B, b[None]])
        Zc = np.append(Zc, c[2])
        n_acc += 1
        filled += _rasterize_cylinder(ph, c, th, radius, length)
    return ph, float(ph.mean()), n_acc


def rsa_spheres(N, radius, frac, seed=0, max_tries=200000):
    """Periodic RSA of spheres; returns (uint8 phase, achieved fraction, n_spheres)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ph = np.zeros((N, N, N), dtype=np.uint8)
    centres = []
    target = frac * N ** 3
    tries = 0
    r_int = int(math.ceil(radius)) + 1
    offs = np.arange(-r_int, r_int + 1)
    while ph.sum(dtype=np.int64) < target and tries < max_tries:
        tries += 1
        c = rng.uniform(0, N, size=3)
        ok = all(np.linalg.norm(_periodic_delta(c - c2, N)) >= 2 * radius + 1 for c2 in centres)
        if not ok:
            continue
        centres.append(c)
        base = np.floor(c).astype(int)
        X, Y, Z = np.meshgrid(base[0] + offs, base[1] + offs, base[2] + offs, indexing="ij")
        d2 = (X + 0.5 - c[0]) ** 2 + (Y + 0.5 - c[1]) ** 2 + (Z + 0.5 - c[2]) ** 2
        m = d2 <= radius * radius
        ph[X[m] % N, Y[m] % N, Z[m] % N] = 1
    return ph, float(ph.mean()), len(centres)


def ode23_batch(n, seed=0):
    """Load-step-like material inputs for the adaptive (ode23) update: z_n
    deviatoric with (z11, z22, g23, g13, g12) ~ U[-0.005, 0.005], eps_n = z_n +
    U[-0.002, 0.002]^6 (trial stresses up to ~2 sigma0 for the matrix law),
    eps = eps_n + U[-0.001, 0.001]^6.  Returns (eps_n, eps, z_n), each (n, 6)."""
    rng = np.random.default_rng(seed)
    y = rng.uniform(-0.005, 0.005, (n, 5))
    zn = np.stack([y[:, 0], y[:, 1], -y[:, 0] - y[:, 1], y[:, 2], y[:, 3], y[:, 4]], axis=1)
    eps_n = zn + rng.uniform(-0.002, 0.002, (n, 6))
    eps = eps_n + rng.uniform(-0.001, 0.001, (n, 6))
    return eps_n, eps, zn


def ramp(n_steps, E_final):
    """E_k = (k / n_steps) E_final, k = 1..n_steps -> (n_steps, 6)."""
    E_final = np.asarray(E_final, dtype=np.float64)
    return np.array([(k / n_steps) * E_final for k in range(1, n_steps + 1)])


# Named workloads ----------------------------------------------------------

# Matrix: elastic-viscoplastic, Norton dissipation (E, nu, sigma0, edot0, n).
MATRIX_16 = (70.0, 0.3, 0.1, 1.0, 5.0)
INCLUSION_16 = (400.0, 0.2)
FIBRE_256 = (72.0, 0.22)
MATRIX_256 = (70.0, 0.3, 0.1, 1.0, 10.0)
# The paper's metal-matrix composite (Table misu_parameters), in GPa and 1/s:
# aluminium (E, nu, sigma_Y, H, edot0, sigma_d, n) and alumina (E, nu).
ALUMINIUM_MS = (55.0, 0.33, 0.025, 1.8, 1.0, 0.130, 3.6)
ALUMINA = (300.0, 0.25)


def sphere_composite_16():
    """16^3 centred sphere (10 %), uniaxial strain ramp to 1 % in 10 steps, h = 0.1."""
    ph = sphere_phase(16, 0.10)
    loads = ramp(10, [0.01, 0, 0, 0, 0, 0])
    return ph, loads, [0.1] * 10


def shear_tension_load(n_steps=20, amp=0.02):
    """E_k = (k/n) amp (1,0,0,0,0,1)/sqrt(2) with engineering g12; h = 0.1."""
    d = np.array([1, 0, 0, 0, 0, 1], dtype=np.float64) / math.sqrt(2.0)
    return ramp(n_steps, amp * d), [0.1] * n_steps


def fibre_composite(N=256, seed=0):
    """RSA cylinders r=6, length 180 (aspect 15), 15 % volume fraction."""
    return rsa_cylinders(N, 6.0, 0.15, min(180.0, 0.7 * N), seed=seed)


def unit_direction(rng):
    """Random unit vector on the Voigt-6 strain space (engineering shears)."""
    d = rng.normal(size=6)
    return d / np.linalg.norm(d)


def _stream_phase(args):
    """Microstructure of one serving job (a process-pool task)."""
    kind, N, frac, seed = args
    if kind == "spheres":
        return rsa_spheres(N, max(2.0, N / 10.0), frac, seed=seed, max_tries=20000)
    return rsa_cylinders(N, max(1.5, N / 32.0), frac, 0.35 * N, seed=seed, max_tries=20000)


def serving_stream(n_jobs=64, seed=0, grids=(32, 64, 96, 128, 192), steps=(5, 20), matrix_n=(3.0, 5.0, 10.0),
                   workers=1):
    """Homogenization jobs of the serving workload.

    Per job: N uniform over ``grids``; microstructure RSA spheres (5-25 %,
    radius max(2, N/10)) or RSA cylinders (10-30 %, radius max(1.5, N/32),
    length 0.35 N; RSA stops after 20000 tries, so dense targets can jam
    below the target -- the achieved fraction is recorded), each with
    probability 1/2; Norton matrix (E=70, nu=0.3,
    sigma0=0.1, edot0=1) with n drawn from ``matrix_n``; inclusion E=400,
    nu=0.2; macro strain ramp along a random unit direction with amplitude
    U[1 %, 2 %] over a step count uniform in ``steps`` (inclusive), h = 0.1.
    The microstructures (each from its own seed) are built by ``workers``
    processes (spawned, so safe after CUDA initialisation); the result does
    not depend on ``workers``.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    specs, jobs = [], []
    for k in range(n_jobs):
        N = int(rng.choice(grids))
        if rng.uniform() < 0.5:
            kind, frac = "spheres", rng.uniform(0.05, 0.25)
        else:
            kind, frac = "cylinders", rng.uniform(0.10, 0.30)
        specs.append((kind, N, frac, seed * 1000 + k))
        n_exp = float(rng.choice(matrix_n))
        amp = rng.uniform(0.01, 0.02)
        n_steps = int(rng.integers(steps[0], steps[1] + 1))
        E = ramp(n_steps, amp * unit_direction(rng))
        jobs.append({"N": N, "kind": kind,
                     "laws": [(1, (70.0, 0.3, 0.1, 1.0, n_exp)), (0, (400.0, 0.2))],
                     "E": E, "h": [0.1] * n_steps})
    if workers > 1:
        import concurrent.futures as cf
        import multiprocessing as mp
        # largest grids first, so the pool's tail is short
        order = sorted(range(n_jobs), key=lambda i: -specs[i][1])
        with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            built = dict(zip(order, ex.map(_stream_phase, [specs[i] for i in order])))
        phases = [built[i] for i in range(n_jobs)]
    else:
        phases = [_stream_phase(sp) for sp in specs]
    for j, (ph, achieved, _) in zip(jobs, phases):
        j["phase"] = ph
        j["fraction"] = achieved
    return jobs
