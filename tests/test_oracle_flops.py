"""Pins of the oracle's algorithmic flop counts (the measurement of the
material update's algorithmic work asks for the flops the method performs per
step of the implicit-Euler update, Sec. 4.1).

Every expected count is derived here by hand from the formulas and the
structure of the constant matrices (P's entries are 0 and +-1; G = P^T W P has
7 nonzero entries; psi_yy = P^T C P = [[4mu, 2mu], [2mu, 4mu]] (+) mu I_3; C
has 12 nonzero entries), so a counter that counts a structural zero, misses a
term or counts a passive constant fails one of them.
"""
import numpy as np
import pytest

import oracle as O
import synth


def hand_counts():
    # psi_y = -P^T C (eps - P y): e = eps - P y (1 add for z33 = -y0-y1, 6 subs),
    # sigma = C e (rows 1-3: 3 mul + 2 add, rows 4-6: 1 mul), P^T sigma (2 adds)
    psi_y = dict(add=1 + 6 + 6 + 2, mul=12)
    # rate v = (y - y_n)/h: 5 sub, 5 div
    rate = dict(add=5, div=5)
    # eqrate: Gv (rows 1, 2: 2 mul + 1 add; rows 3-5: 1 mul), q = v.Gv (5 mul, 4 add), sqrt
    eqrate = dict(add=2 + 4, mul=7 + 5, sqrt=1)
    # phi_v = (sigma0 edot0^(-1/n)) s^(1/n-1) Gv: 1 pow, 1 mul, 5 mul
    phi_v = dict(mul=6, pow=1)
    residual = add(psi_y, rate, eqrate, phi_v, dict(add=5))
    # phi_vv = c1 G + c2 Gv Gv^T: 2 pow, 2 mul (constants times powers),
    # 7 mul + 7 add where G != 0, 2 mul per entry (25); K = psi_yy + phi_vv/h: 25 div, 7 add
    K = add(rate, eqrate, dict(mul=2 + 7 + 50, add=7 + 7, div=25, pow=2))
    # dense 5x5 Cholesky: factor 20 mul + 20 sub, 5 sqrt, 10 div; two substitutions 20 mul + 20 sub + 10 div
    factor = dict(mul=20, add=20, sqrt=5, div=10)
    subst = dict(mul=20, add=20, div=10)
    newton = add(residual, K, factor, subst, dict(add=5))
    # predictor: psi_y(eps, y_n), then substitutions with the block factor of
    # psi_yy (2x2 block: 1 mul + 1 sub + 2 div per sweep; 3 diagonal: 1 div per sweep)
    predictor = add(psi_y, dict(mul=2, add=2, div=10))
    # one line-search step: y_n + theta d (5 mul, 5 add), R, K, g = d.R (5 mul, 4 add),
    # g' = d^T K d (50 mul, 24 add), theta - g/g' (1 div, 1 sub)
    line = add(dict(mul=5, add=5), residual, K, dict(mul=5, add=4), dict(mul=50, add=24), dict(div=1, add=1))
    # stress: z = P y (1 add), e = eps - P y (7 add), sigma = C e (12 mul, 6 add)
    stress = dict(add=14, mul=12)
    # tangent: K, one factor, 6 column solves with a passive right-hand side
    # ((P^T C)_j has 2 or 3 nonzero entries: the forward sweep skips the work
    # on leading zeros), (C P) dy/deps per column and the subtraction
    return dict(residual=residual, newton=newton, predictor=predictor, line=line, stress=stress, subst=subst, K=K,
                factor=factor)


def add(*ds):
    out = {k: 0 for k in O.FLOP_KINDS}
    for d in ds:
        for k, v in d.items():
            out[k] += v
    return out


@pytest.fixture(scope="module")
def counted():
    prm = (70.0, 0.3, 0.1, 1.0, 5.0)
    eps, zn = synth.material_batch(64, seed=3)
    s, z, info = O.update(O.KIND_NORTON, prm, eps, zn, 0.01, info=True)
    i = int(np.argmax(np.abs(z - zn).sum(axis=1)))  # a flowing voxel
    y = z[i][[0, 1, 3, 4, 5]]
    return O.flop_pieces(prm, eps[i], zn[i], y, 0.01)


@pytest.mark.parametrize("piece", ["residual", "newton", "predictor", "line", "stress", "subst"])
def test_flop_counts_equal_the_hand_count(counted, piece):
    assert counted[piece] == add(hand_counts()[piece]), (piece, counted[piece])


def test_flop_counts_do_not_depend_on_the_state():
    """Counts follow the formulas' structure, not the values: two flowing
    voxels, two step sizes and exponents give the same numbers."""
    eps, zn = synth.material_batch(8, seed=9)
    seen = []
    for n_exp, h in ((5.0, 0.01), (3.0, 0.1)):
        prm = (70.0, 0.3, 0.1, 1.0, n_exp)
        s, z = O.update(O.KIND_NORTON, prm, eps, zn, h)
        for i in (0, 5):
            seen.append(O.flop_pieces(prm, eps[i], zn[i], z[i][[0, 1, 3, 4, 5]], h))
    assert all(c == seen[0] for c in seen)


def test_flop_pieces_refuse_a_state_without_flow():
    eps, zn = synth.material_batch(1, seed=1)
    with pytest.raises(ValueError):
        O.flop_pieces((70.0, 0.3, 0.1, 1.0, 5.0), eps[0], zn[0], zn[0][[0, 1, 3, 4, 5]], 0.01)


def test_tangent_count_is_bounded_by_its_pieces(counted):
    """The tangent is K, one factor and six solves plus (C P) dy: at least K +
    factor, at most K + factor + 6 full substitutions + 6 x (6x5 products)."""
    h = hand_counts()
    t = counted["tangent"]
    lo = add(h["K"], h["factor"])
    hi = add(h["K"], h["factor"], *[h["subst"]] * 6, *[dict(mul=30, add=30)] * 6)
    for k in O.FLOP_KINDS:
        assert lo[k] <= t[k] <= hi[k], (k, t[k], lo[k], hi[k])
