"""Shock tube at xi = 1 (the RSST reduces to conservative Euler, Sec. 3.2)
against the exact Riemann solution; the exact solver itself is pinned to the
star state printed in the textbook literature (tests/golden)."""
import json
import os

import numpy as np
import pytest

from oracle import riemann_exact as rx
from oracle import rsst_oracle as ro
from oracle.workload import problem_from
from paper_1812_04135_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden", "sod_star_state.json")


def test_exact_riemann_star_state_matches_textbook():
    g = json.load(open(GOLD))
    L, R, S = g["left"], g["right"], g["star"]
    p, u = rx.star_state(L["rho"], L["u"], L["p"], R["rho"], R["u"], R["p"], g["gamma"])
    rl, rr = rx.star_densities(L["rho"], L["p"], R["rho"], R["p"], p, g["gamma"])
    tol = g["abs_tol"]
    assert abs(p - S["p"]) < tol and abs(u - S["u"]) < tol
    assert abs(rl - S["rho_left"]) < tol and abs(rr - S["rho_right"]) < tol


def _sod_error(n, t_end=0.2):
    w = inputs.sod_1d(n)
    prob, U = problem_from(w)
    t = 0.0
    while t < t_end - 1e-14:
        dt = min(ro.cfl_dt(U, prob), t_end - t)
        U = ro.ssp_rk2_step(U, dt, prob)
        t += dt
    x = (np.arange(n) + 0.5) / n
    exact = np.array([rx.sample((xi - 0.5) / t_end, 1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 1.4)[0] for xi in x])
    return float(np.mean(np.abs(U[0].numpy() - exact)))


def test_sod_converges_to_exact_solution():
    e1, e2, e3 = _sod_error(100), _sod_error(200), _sod_error(400)
    assert e3 < e2 < e1
    assert e2 < 0.02
    order = np.log2(e2 / e3)
    assert 0.6 < order < 1.4           # discontinuities limit a 2nd-order scheme to ~1st order in L1
