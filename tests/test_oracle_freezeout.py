"""Pins of the freeze-out hypersurface oracle (oracle/clv_freezeout.c,
readings F1-F6 of the surface elements dSigma_mu of Eq. (cooper_frye)).

Everything here is fixed by geometry, not by the oracle:
  - affine level sets are reproduced exactly by the piecewise-linear
    interpolant, so their dSigma_mu sums are closed-form integrals;
  - inside one 4-simplex the coarea formula gives the piece in closed form:
    dSigma_mu = -grad_mu f vol4(S) M(0), M the Curry-Schoenberg B-spline with
    the vertex values as knots (the density of f over the simplex);
  - a closed level set has sum dSigma_mu = 0 (Cartesian) and, with the Milne
    weight tau, sum dSigma_i = 0 and sum dSigma_tau = the enclosed 4-volume;
  - affine fields are interpolated exactly;
  - the crossed hypercubes are those whose 16 corners straddle eps_f.
"""
import itertools
import math

import numpy as np
import pytest

import oracle


def _coords(n, d):
    return (np.arange(n) - 0.5 * (n - 1)) * d


def _grid(shape, d):
    x, y, z = (_coords(n, dd) for n, dd in zip(shape, d))
    return np.meshgrid(x, y, z, indexing="ij")


SHAPE = (7, 6, 5)
D = (0.3, 0.25, 0.2)
L = [(n - 1) * d for n, d in zip(SHAPE, D)]


def check_planar_tau(plant=0, cartesian=False):
    tau0, tau1, A, B, ef = 1.3, 1.7, 2.0, 0.5, 1.1
    e0, e1 = np.full(SHAPE, A), np.full(SHAPE, B)
    rec, cube, n = oracle.freezeout(e0, e1, ef, *D, tau0, tau1, cartesian=cartesian, plant=plant)
    assert n == np.prod([s - 1 for s in SHAPE])
    tstar = tau0 + (A - ef) / (A - B) * (tau1 - tau0)
    w = 1.0 if cartesian else tstar
    S = rec[:, :4].sum(axis=0)
    np.testing.assert_allclose(S[0], w * L[0] * L[1] * L[2], rtol=1e-13)
    assert np.abs(S[1:]).max() <= 1e-13 * S[0]
    np.testing.assert_allclose(rec[:, 4], tstar, rtol=1e-14)


def _planar_axis(axis, plant=0, cartesian=False, slope_tau=0.0):
    """eps = ef + g (c* - c) - a (tau - tau*) along spatial axis `axis`."""
    tau0, tau1, ef, g = 0.8, 1.4, 1.0, 2.0
    X = _grid(SHAPE, D)
    cstar = 0.37 * L[axis] / 2
    taus = 0.5 * (tau0 + tau1)
    e = [ef + g * (cstar - X[axis]) - slope_tau * (t - taus) for t in (tau0, tau1)]
    rec, _, n = oracle.freezeout(e[0], e[1], ef, *D, tau0, tau1, cartesian=cartesian, plant=plant)
    w = (tau1 - tau0) if cartesian else 0.5 * (tau1 ** 2 - tau0 ** 2)
    other = [L[a] for a in range(3) if a != axis]
    want = np.zeros(4)
    want[1 + axis] = w * other[0] * other[1]
    want[0] = slope_tau / g * want[1 + axis]
    S = rec[:, :4].sum(axis=0)
    np.testing.assert_allclose(S, want, rtol=1e-12, atol=1e-13 * want[1 + axis])
    # the element positions lie on the plane
    c = rec[:, 5 + axis]
    np.testing.assert_allclose(g * (cstar - c) - slope_tau * (rec[:, 4] - taus), 0.0, atol=1e-12)
    return n


def check_planar_axes(plant=0):
    for axis in range(3):
        for cart in (False, True):
            _planar_axis(axis, plant, cart)
            _planar_axis(axis, plant, cart, slope_tau=0.9)


def test_planar_level_set_in_time_gives_the_tau_slab():
    check_planar_tau()
    check_planar_tau(cartesian=True)


def test_planar_level_sets_in_space_and_oblique():
    check_planar_axes()


def _bspline_density(t, knots):
    """Curry-Schoenberg B-spline of degree 3 on 5 distinct knots, normalised
    to unit integral: the density of a linear function of a uniform point of
    a 4-simplex whose vertex values are the knots."""
    s = 0.0
    for i, fi in enumerate(knots):
        den = np.prod([fi - fj for j, fj in enumerate(knots) if j != i])
        s += max(fi - t, 0.0) ** 3 / den
    return 4.0 * s


def check_simplices(plant=0, seed=11):
    rng = np.random.default_rng(seed)
    h = (0.07, 0.3, 0.25, 0.2)
    vol4 = np.prod(h) / 24.0
    crossed = 0
    for trial in range(30):
        e0 = rng.uniform(-1, 1, (2, 2, 2))
        e1 = rng.uniform(-1, 1, (2, 2, 2))
        ef = rng.uniform(-0.3, 0.3)
        for s, perm in enumerate(itertools.permutations(range(4))):
            v = [0]
            for a in perm:
                v.append(v[-1] | (1 << a))
            f = [(e1 if q & 1 else e0)[q >> 1 & 1, q >> 2 & 1, q >> 3 & 1] - ef for q in v]
            grad = np.zeros(4)
            for m, a in enumerate(perm):
                grad[a] = (f[m + 1] - f[m]) / h[a]
            want = -grad * vol4 * _bspline_density(0.0, f)
            got = oracle.freezeout_simplex(e0, e1, ef, *h[1:], 1.0, 1.0 + h[0], 0, 0, 0, s,
                                           cartesian=True, plant=plant)
            crossed += bool(np.any(got != 0))
            np.testing.assert_allclose(got, want, rtol=1e-8, atol=1e-9 * vol4 * np.abs(grad).max())
    assert crossed > 200


def test_each_simplex_matches_the_coarea_closed_form():
    check_simplices()


def _ball(n, R, cartesian, plant=0):
    """Level set 1 - r^2/R^2 = 1/2 of a 4-ball centred in the box, found
    slice pair by slice pair over n+1 time slices: the union is closed."""
    shape = (n, n, n)
    h = 2.6 * R / (n - 1)
    tc = 3.0 * R
    taus = tc + (np.arange(n) - 0.5 * (n - 1)) * h
    X, Y, Z = _grid(shape, (h, h, h))
    eps = [1.0 - ((t - tc) ** 2 + X ** 2 + Y ** 2 + Z ** 2) / R ** 2 for t in taus]
    S = np.zeros(4)
    A = 0.0
    cnt = 0
    for a in range(n - 1):
        rec, _, m = oracle.freezeout(eps[a], eps[a + 1], 0.5, h, h, h, taus[a], taus[a + 1],
                                     cartesian=cartesian, plant=plant)
        S += rec[:, :4].sum(axis=0)
        A += np.sqrt((rec[:, :4] ** 2).sum(axis=1)).sum()
        cnt += m
    return S, A, cnt


def check_closed_surface(plant=0):
    """Sum dSigma = 0 exactly (Cartesian); with the Milne weight the spatial
    sums vanish and dSigma_tau sums to the enclosed 4-volume, which converges
    at second order to the ball (the interpolant of the concave profile lies
    below it, so the region is smaller by O(h^2))."""
    R = 1.0
    r = R / math.sqrt(2.0)      # radius of the level 1/2
    vol = math.pi ** 2 * r ** 4 / 2
    errs = []
    for n in (9, 17):
        S, A, cnt = _ball(n, R, cartesian=True, plant=plant)
        assert cnt > 300
        assert np.abs(S).max() <= 1e-12 * A
        S, A, _ = _ball(n, R, cartesian=False, plant=plant)
        assert np.abs(S[1:]).max() <= 1e-12 * A
        errs.append(abs(S[0] / vol - 1))
    assert errs[1] < 0.08 and errs[0] / errs[1] > 3.3, errs


def test_closed_level_set_sums_to_zero_and_encloses_the_ball():
    check_closed_surface()


def test_closed_surface_area_converges_to_the_three_sphere():
    r = 1.0 / math.sqrt(2.0)
    area = 2 * math.pi ** 2 * r ** 3
    errs = [abs(_ball(n, 1.0, True)[1] / area - 1) for n in (9, 17)]
    assert errs[1] < 0.05 and errs[0] / errs[1] > 3.3, errs


def test_affine_fields_are_interpolated_exactly():
    rng = np.random.default_rng(5)
    tau0, tau1 = 2.0, 2.3
    X = _grid(SHAPE, D)
    e0 = 1.0 + 0.4 * rng.normal(size=SHAPE)
    e1 = 1.0 + 0.4 * rng.normal(size=SHAPE)
    coef = rng.normal(size=(13, 5))
    f = [np.stack([c[0] + c[1] * t + c[2] * X[0] + c[3] * X[1] + c[4] * X[2] for c in coef])
         for t in (tau0, tau1)]
    rec, _, n = oracle.freezeout(e0, e1, 1.0, *D, tau0, tau1, f[0], f[1])
    assert n > 50
    pos = rec[:, 4:8]
    want = coef[:, 0][None] + pos @ coef[:, 1:].T
    np.testing.assert_allclose(rec[:, 9:], want, atol=1e-12)
    np.testing.assert_allclose(rec[:, 8], np.sqrt(1 + (want[:, :3] ** 2).sum(axis=1)), rtol=1e-14)


def test_crossed_hypercubes_are_the_straddling_ones_in_order():
    rng = np.random.default_rng(8)
    shape = (9, 7, 6)
    e0 = rng.uniform(0, 1, shape)
    e1 = rng.uniform(0, 1, shape)
    ef = 0.6
    rec, cube, n = oracle.freezeout(e0, e1, ef, 0.2, 0.2, 0.2, 1.0, 1.1)
    corners = [e[a:a + shape[0] - 1, b:b + shape[1] - 1, c:c + shape[2] - 1]
               for e in (e0, e1) for a in (0, 1) for b in (0, 1) for c in (0, 1)]
    mx, mn = np.max(corners, axis=0), np.min(corners, axis=0)
    want = np.flatnonzero(((mx >= ef) & (mn < ef)).ravel())
    assert n == len(want)
    np.testing.assert_array_equal(cube, want)
    # a smaller capacity keeps the first records and still counts them all
    rec2, cube2, n2 = oracle.freezeout(e0, e1, ef, 0.2, 0.2, 0.2, 1.0, 1.1, capacity=17)
    assert n2 == n and len(rec2) == 17
    np.testing.assert_array_equal(rec2, rec[:17])
    # nothing crosses when every corner is on one side
    for v in (0.59, 0.6):
        assert oracle.freezeout(np.full(shape, 1.0), np.full(shape, 1.0), v, 0.2, 0.2, 0.2, 1.0, 1.1)[2] == 0
    assert oracle.freezeout(e0, e1, 1.01, 0.2, 0.2, 0.2, 1.0, 1.1)[2] == 0


def test_bad_grid_is_rejected():
    with pytest.raises(ValueError):
        oracle.freezeout(np.zeros((1, 3, 3)), np.zeros((1, 3, 3)), 0.5, 0.2, 0.2, 0.2, 1.0, 1.1)
    with pytest.raises(ValueError):
        oracle.freezeout(np.zeros((3, 3, 3)), np.zeros((3, 3, 3)), 0.5, 0.2, 0.2, 0.2, 1.0, 1.0)
