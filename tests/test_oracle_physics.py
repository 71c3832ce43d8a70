"""Physics pins of the oracle: the exact Sod solution (the RiemannProblem of
Sec. 3, Fig. 1) and convergence orders on a smooth wave.

The exact Riemann solver in ``exact_riemann.py`` is itself pinned to the
textbook star state in ``golden/sod_star_toro.txt``.
"""
import math
import os

import numpy as np
import pytest

import exact_riemann as er
from paper_1812_07977_gb300 import problems

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sod_star_toro.txt")
L, R = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)


def _golden():
    vals = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    return vals


def test_exact_solver_matches_textbook_star_state():
    g = _golden()
    ps, us = er.star_state(L, R)
    assert abs(ps - g["p_star"]) < 5e-6
    assert abs(us - g["u_star"]) < 5e-6
    rho_l = er.sample(0.5 * us, L, R)[0]      # inside the left star region
    rho_r = er.sample(1.2 * us, L, R)[0]      # between contact and shock
    assert abs(rho_l - g["rho_star_left"]) < 5e-6
    assert abs(rho_r - g["rho_star_right"]) < 5e-6


def test_exact_solver_wave_speeds():
    ps, us = er.star_state(L, R)
    cl = math.sqrt(1.4)
    # rarefaction head at -c_L, shock at u_R + c_R sqrt((g+1)/(2g) p*/p_R + (g-1)/(2g))
    assert er.sample(-cl - 1e-9, L, R) == L
    assert er.sample(-cl + 1e-3, L, R)[0] < 1.0
    cr = math.sqrt(1.4 * 0.1 / 0.125)
    s_shock = cr * math.sqrt(2.4 / 2.8 * ps / 0.1 + 0.4 / 2.8)
    assert abs(s_shock - 1.7522) < 1e-4
    assert er.sample(s_shock + 1e-9, L, R) == R
    assert er.sample(s_shock - 1e-9, L, R)[2] == pytest.approx(ps, rel=1e-12)


def _sod_l1(orc, n, theta, t=0.2):
    m = orc.mesh(n, 1, 1, theta=theta)
    U = orc.ghosted_from_interior(m, problems.riemann_planar(n, 1, 1))
    orc.evolve(m, U, 0.4, t_end=t)
    ex = er.cell_average_density(n, t, L, R, sub=16)
    return np.abs(orc.interior(U)[0, 0, 0] - ex).mean(), orc.interior(U)


def test_sod_converges_and_second_order_beats_first(orc):
    ns = [32, 64, 128, 256]
    e2 = [_sod_l1(orc, n, 2.0)[0] for n in ns]
    e0 = [_sod_l1(orc, n, 0.0)[0] for n in ns]
    assert all(a > b for a, b in zip(e2, e2[1:])), e2
    assert all(a > b for a, b in zip(e0, e0[1:])), e0
    assert all(a < b for a, b in zip(e2, e0)), (e2, e0)
    r2 = math.log2(e2[0] / e2[-1]) / (len(ns) - 1)
    r0 = math.log2(e0[0] / e0[-1]) / (len(ns) - 1)
    assert r2 > r0
    # discontinuous solution: L1 order <= 1; first order smears the contact
    assert 0.8 < r2 < 1.2 and 0.4 < r0 < 0.8, (r2, r0)
    assert e2[-1] < 3e-3


def test_sod_star_plateau(orc):
    # Fig. 1 analogue: 1D Sod at 128 cells and t = 0.25
    _, U = _sod_l1(orc, 128, 2.0, t=0.25)
    ps, us = er.star_state(L, R)
    x = problems.cell_centres(128)
    rho, u = U[0, 0, 0], U[1, 0, 0] / U[0, 0, 0]
    p = 0.4 * (U[4, 0, 0] - 0.5 * rho * u * u)
    mid = (x > 0.5 + 0.25 * (us * 0.25)) & (x < 0.5 + 0.75 * us * 0.25)
    assert mid.sum() >= 3
    assert np.all(np.abs(p[mid] - ps) < 0.01 * ps)
    assert np.all(np.abs(u[mid] - us) < 0.01 * us)


def _wave_l1(orc, n, theta):
    m = orc.mesh(n, 1, 1, theta=theta, bc=(1, 1, 1))
    U0 = problems.entropy_wave_1d(n)
    U = orc.ghosted_from_interior(m, U0)
    orc.evolve(m, U, 0.4, t_end=1.0)   # one period: exact solution = initial
    return np.abs(orc.interior(U)[0] - U0[0]).mean()


def test_smooth_wave_orders(orc):
    ns = [32, 64, 128, 256]
    e2 = [_wave_l1(orc, n, 2.0) for n in ns]
    e0 = [_wave_l1(orc, n, 0.0) for n in ns]
    r2 = math.log2(e2[-2] / e2[-1])
    r0 = math.log2(e0[-2] / e0[-1])
    assert 1.8 < r2 < 2.2, e2
    assert 0.8 < r0 < 1.2, e0


def test_smooth_wave_3d_oblique(orc):
    # the 3D wave along (1,1,1): at t = 1/3 the exact solution is the initial data
    errs = []
    for n in (8, 16):
        m = orc.mesh(n, n, n, bc=(1, 1, 1))
        U0 = problems.entropy_wave_3d(n)
        U = orc.ghosted_from_interior(m, U0)
        orc.evolve(m, U, 0.4, t_end=1.0 / 3.0)
        errs.append(np.abs(orc.interior(U)[0] - U0[0]).mean())
    assert errs[1] < errs[0] / 2.5, errs
