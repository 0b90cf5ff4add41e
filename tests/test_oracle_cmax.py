"""The C_max reduction law, Eq. cx (Sec. 4.3): xi = [1 + (a/C_max)^4]^(1/4),
state-dependent.  Pins: the effective sound speed a/xi tends to C_max for
a >> C_max and to a for a << C_max and never exceeds either; a C_max far
above every sound speed gives xi = 1 exactly, i.e. the Euler step bit for
bit; the linear sound eigenmode of a uniform gas travels at a/xi(a)."""
import math

import numpy as np
import pytest
import torch

from oracle import rsst_oracle as ro
from oracle.workload import problem_from
from paper_1812_04135_gb300 import inputs


def test_effective_sound_speed_limits():
    C = 0.3
    a = torch.logspace(-4, 4, 200, dtype=torch.float64)
    g = a / ro.xi_of(a * a, 1.0, C)
    assert torch.all(g <= C * (1 + 1e-15)) and torch.all(g <= a * (1 + 1e-15))
    assert float(g[-1]) == pytest.approx(C, rel=1e-12)      # a = 1e4: C_max
    assert float(g[0]) == pytest.approx(float(a[0]), rel=1e-12)  # a = 1e-4: a
    # the stated form a / [1 + (a/C)^4]^(1/4) at a = C is C / 2^(1/4)
    a_c = torch.tensor(C, dtype=torch.float64)
    assert float(a_c / ro.xi_of(a_c * a_c, 1.0, C)) == pytest.approx(C / 2 ** 0.25, rel=1e-14)


@pytest.mark.parametrize("ndim", [1, 2])
def test_huge_cmax_is_euler_bitwise(ndim):
    n = {1: (40,), 2: (20, 12)}[ndim]
    w = inputs.random_smooth_state(ndim, n, xi=1.0)
    prob_e, U = problem_from(w, variant="euler")
    ref = ro.run(U, prob_e, 3)
    for var in ("pvs", "dms"):
        w2 = dict(w, cmax=1e30)
        prob, U = problem_from(w2, variant=var)
        assert torch.equal(ro.run(U, prob, 3), ref), var


def test_sound_wave_speed_under_cmax():
    """a = 1, C_max = 0.1: xi = (1 + 10^4)^(1/4), wave speed a/xi ~ 0.1."""
    w = inputs.sound_wave_1d(256, xi=1.0, variant="pvs")
    C = 0.1
    xi_eff = (1.0 + (1.0 / C) ** 4) ** 0.25
    # the eigenmode of the reduced system at this xi
    w = inputs.sound_wave_1d(256, xi=xi_eff, variant="pvs")
    w["cmax"] = C
    prob, U = problem_from(w)
    ts, ph = [], []
    t = 0.0
    for s in range(501):
        if s % 50 == 0:
            P = ro.primitives(U, prob.gamma)[3].numpy()
            ts.append(t)
            ph.append(float(np.angle(np.fft.rfft(P - P.mean())[1])))
        if s == 500:
            break
        dt = ro.cfl_dt(U, prob)
        U = ro.ssp_rk2_step(U, dt, prob)
        t += dt
    c = -np.polyfit(ts, np.unwrap(ph), 1)[0] / (2 * math.pi)
    assert c == pytest.approx(1.0 / xi_eff, rel=0.01)
