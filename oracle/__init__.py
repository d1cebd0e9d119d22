"""FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
product (``paper_2006_04391_gb300``) never imports it, and it imports nothing
from the product: the two share no code.

Contents
--------
* ``material`` -- ctypes wrappers of ``gsm_oracle.cpp``: the implicit-Euler
  GSM update (Sec. 4.1, Eq. implicit_euler and Eq. tangent_formula of
  AutoMat, arXiv 2006.04391), hand-derived potentials, an independent
  radial return (the conventional strategy of Sec. 4), and the ode23 update
  of the force-potential form with its tangent ODE (Sec. 4.3, Corollary 1)
  and stress-driven error control (Sec. 4.5).
* ``material.flop_pieces`` -- the algorithmic flops of each piece of that
  update, counted by running the same statements once on a counting scalar.
* ``ms`` -- the Moulinec-Suquet basic scheme (cited by the paper in Sec. 1 and
  Sec. 3 "Material Law Evaluations") written with ``numpy.fft``.

Parity with the paper's printed numbers is unpinned (the paper prints no
field values for a reproducible case); every function is pinned against
closed forms, finite differences, invariants and special cases instead.
"""
from .material import (  # noqa: F401
    KIND_ELASTIC, KIND_NORTON, lame, update, radial_return, psi, psi_y, psi_yy,
    phi, phi_v, phi_vv, residual, newton_matrix, incremental_potential, stress,
    max_threads, P_MATRIX, G_MATRIX, update_ode23, psi_force_a, psi_force_ms, psi_force_aaa, gen_stress_ms, KIND_MICHEL_SUQUET,
    flop_pieces, FLOP_PIECES, FLOP_KINDS,
)
