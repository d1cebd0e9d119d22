"""Input recipes: determinism, volume fractions, non-overlap, deviatoric z_n."""
import math

import numpy as np

import synth


def test_material_batch_is_seeded_and_deviatoric():
    a = synth.material_batch(1000, seed=5)
    b = synth.material_batch(1000, seed=5)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    eps, zn = a
    assert np.max(np.abs(eps)) <= 0.02 and np.max(np.abs(zn[:, [0, 1, 3, 4, 5]])) <= 0.005
    assert np.max(np.abs(zn[:, :3].sum(axis=1))) < 1e-18


def test_sphere_fraction_close_to_target():
    ph = synth.sphere_phase(64, 0.2)
    assert abs(ph.mean() - 0.2) < 0.01
    assert ph[32, 32, 32] == 1 and ph[0, 0, 0] == 0


def test_rsa_cylinders_fraction_and_separation():
    N, r, L = 48, 2.0, 30.0
    ph, frac, nf = synth.rsa_cylinders(N, r, 0.10, L, seed=3)
    assert frac >= 0.10 and frac < 0.13 and nf >= 3
    ph2, frac2, _ = synth.rsa_cylinders(N, r, 0.10, L, seed=3)
    assert np.array_equal(ph, ph2)


def test_rsa_spheres_fraction():
    ph, frac, n = synth.rsa_spheres(40, 4.0, 0.15, seed=2)
    assert 0.15 <= frac < 0.2 and n >= 5


def test_segment_distance_helper():
    d = synth._seg_seg_dist_2d(np.array([0.0, 0]), np.array([1.0, 0]), np.array([0.0, 2]), np.array([1.0, 2]))
    assert abs(d - 2.0) < 1e-15
    d = synth._seg_seg_dist_2d(np.array([0.0, 0]), np.array([2.0, 2]), np.array([0.0, 2]), np.array([2.0, 0]))
    assert d == 0.0
    d = synth._seg_seg_dist_2d(np.array([0.0, 0]), np.array([1.0, 0]), np.array([2.0, 1]), np.array([3.0, 1]))
    assert abs(d - math.sqrt(2.0)) < 1e-15
