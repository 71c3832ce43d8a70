"""Pins of the oracle's single-state pieces: cons<->prim, limiter, HLL.

Each check is independent of the oracle's own formulas: round trips, exact
special cases of the limiter, consistency/upwinding of the HLL flux, and a
textbook-form HLL (Toro, Ch. 10, the S_L / S_R branch form) written here.
"""
import math

import numpy as np
import pytest

from paper_1812_07977_gb300 import problems

G = 1.4


def test_cons_prim_round_trip(orc):
    states = problems.random_states(seed=7, n=2000, vmax=1.0)
    for w in states:
        u = orc.prim_to_cons(G, w)
        w2 = orc.cons_to_prim(G, u)
        # moderate Mach numbers: a few ulp of each component's scale
        np.testing.assert_allclose(w2[0], w[0], rtol=0, atol=0)
        np.testing.assert_allclose(w2[1:4], w[1:4], rtol=4e-16, atol=4e-16 * abs(w[1:4]).max())
        assert abs(w2[4] - w[4]) <= 1e-13 * (w[4] + w[0] * (w[1:4] ** 2).sum())


def test_cons_prim_closed_form(orc):
    # rho=2, v=(1,-2,3), p=0.8:  E = 0.8/0.4 + 0.5*2*14 = 16
    u = orc.prim_to_cons(G, [2.0, 1.0, -2.0, 3.0, 0.8])
    np.testing.assert_allclose(u, [2.0, 2.0, -4.0, 6.0, 16.0], rtol=2e-16)
    w = orc.cons_to_prim(G, [2.0, 2.0, -4.0, 6.0, 16.0])
    np.testing.assert_allclose(w, [2.0, 1.0, -2.0, 3.0, 0.8], rtol=1e-15)


def test_minmod_special_cases(orc):
    assert orc.minmod3(1.0, 2.0, 3.0) == 1.0
    assert orc.minmod3(3.0, 0.5, 2.0) == 0.5
    assert orc.minmod3(-1.0, -2.0, -0.25) == -0.25
    assert orc.minmod3(1.0, -2.0, 3.0) == 0.0
    assert orc.minmod3(0.0, 2.0, 3.0) == 0.0
    assert orc.minmod3(-0.0, -2.0, -3.0) == 0.0
    assert math.copysign(1.0, orc.minmod3(1.0, -1.0, 1.0)) == 1.0   # +0
    assert orc.minmod3(float("nan"), 1.0, 1.0) == 0.0


@pytest.mark.parametrize("theta", [1.0, 1.5, 2.0])
def test_limiter_linear_data_gives_centred_slope(orc, theta):
    # linear data: equal one-sided differences -> the slope is that difference
    for d in [1e-8, 0.3, -2.5, 7.0]:
        assert orc.limited_slope(theta, d, d) == d


def test_limiter_extremum_and_first_order(orc):
    assert orc.limited_slope(2.0, 0.3, -0.1) == 0.0      # local extremum
    assert orc.limited_slope(0.0, 0.3, 0.4) == 0.0       # theta=0: first order
    # MC picks the centred difference when the one-sided ones are close
    assert orc.limited_slope(2.0, 1.0, 2.0) == 1.5
    # ... and 2x the smaller one-sided difference near a steep jump
    assert orc.limited_slope(2.0, 0.1, 5.0) == 0.2
    # minmod (theta=1) takes the smaller one-sided difference
    assert orc.limited_slope(1.0, 0.1, 5.0) == 0.1


def _euler_flux(axis, w):
    rho, v, p = w[0], np.array(w[1:4]), w[4]
    E = p / (G - 1.0) + 0.5 * rho * float(v @ v)
    u = v[axis]
    f = np.empty(5)
    f[0] = rho * u
    f[1:4] = rho * u * v
    f[1 + axis] += p
    f[4] = (E + p) * u
    U = np.array([rho, *(rho * v), E])
    return f, U


def _hll_textbook(axis, wl, wr):
    """Toro Ch. 10: F = F_L if S_L >= 0; F_R if S_R <= 0; else
    (S_R F_L - S_L F_R + S_L S_R (U_R - U_L)) / (S_R - S_L), with Davis
    bounds S_L = min(u_L - c_L, u_R - c_R), S_R = max(u_L + c_L, u_R + c_R)."""
    fl, ul = _euler_flux(axis, wl)
    fr, ur = _euler_flux(axis, wr)
    cl = math.sqrt(G * wl[4] / wl[0])
    cr = math.sqrt(G * wr[4] / wr[0])
    sl = min(wl[1 + axis] - cl, wr[1 + axis] - cr)
    sr = max(wl[1 + axis] + cl, wr[1 + axis] + cr)
    if sl >= 0.0:
        return fl
    if sr <= 0.0:
        return fr
    return (sr * fl - sl * fr + sl * sr * (ur - ul)) / (sr - sl)


def test_hll_consistency(orc):
    states = problems.random_states(seed=11, n=500, vmax=2.0)
    for axis in range(3):
        for w in states:
            f = orc.hll_flux(axis, G, w, w)
            fe, _ = _euler_flux(axis, w)
            scale = np.abs(fe).max() + w[4]
            np.testing.assert_allclose(f, fe, rtol=0, atol=2e-15 * scale)


def test_hll_supersonic_upwinding(orc):
    # both states moving right faster than sound: flux = F(left) up to rounding
    wl = np.array([1.0, 5.0, 0.3, -0.2, 1.0])
    wr = np.array([0.5, 4.0, 0.1, 0.4, 0.7])
    f = orc.hll_flux(0, G, wl, wr)
    fe, _ = _euler_flux(0, wl)
    np.testing.assert_allclose(f, fe, rtol=1e-15, atol=1e-15)
    # mirrored: moving left -> flux = F(right)
    wl2 = wl * np.array([1, -1, 1, 1, 1])
    wr2 = wr * np.array([1, -1, 1, 1, 1])
    f = orc.hll_flux(0, G, wr2, wl2)
    fe, _ = _euler_flux(0, wl2)
    np.testing.assert_allclose(f, fe, rtol=1e-15, atol=1e-15)


def test_hll_matches_textbook_form(orc):
    a = problems.random_states(seed=21, n=10000, vmax=1.5)
    b = problems.random_states(seed=22, n=10000, vmax=1.5)
    worst = 0.0
    for axis in range(3):
        for wl, wr in zip(a[axis::3], b[axis::3]):
            f = orc.hll_flux(axis, G, wl, wr)
            ft = _hll_textbook(axis, wl, wr)
            scale = max(np.abs(ft).max(), np.abs(_euler_flux(axis, wl)[1]).max(),
                        np.abs(_euler_flux(axis, wr)[1]).max())
            worst = max(worst, np.abs(f - ft).max() / scale)
    assert worst < 1e-14, worst


def test_hll_mirror_symmetry_is_exact(orc):
    # reflecting the normal axis swaps the sides and negates the normal
    # velocity; the HLL flux then changes sign in every component but the
    # normal momentum -- exactly, since every operation is sign-symmetric
    a = problems.random_states(seed=5, n=300)
    b = problems.random_states(seed=6, n=300)
    flip = np.array([1.0, -1.0, 1.0, 1.0, 1.0])
    sgn = np.array([-1.0, 1.0, -1.0, -1.0, -1.0])
    for wl, wr in zip(a, b):
        f = orc.hll_flux(0, G, wl, wr)
        fm = orc.hll_flux(0, G, wr * flip, wl * flip)
        assert np.array_equal(fm, sgn * f)
