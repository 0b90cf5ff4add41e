"""Oracle pins from the dynamics of the 1D periodic ideal gas (gamma = 5/3,
N = 256): the sound eigenmode travels at a/xi while the entropy (contact)
wave keeps the flow speed (Sec. 2.1, Sec. 3.1); pressure and velocity stay
uniform across an advected density jump in the pressure-reduced forms and at
xi = 1, while the density-reduced forms create the spurious pressure rate of
Eq. dvs_pr (Sec. 2.2)."""
import math

import numpy as np
import pytest
import torch

from oracle import rsst_oracle as ro
from oracle.workload import problem_from
from paper_1812_04135_gb300 import inputs

G = 5.0 / 3.0


def _mode1_phase(q):
    return float(np.angle(np.fft.rfft(q)[1]))


def _phase_speed(w, var, nsteps, every, field):
    prob, U = problem_from(w, variant=var)
    ts, ph = [], []
    t = 0.0
    for s in range(nsteps + 1):
        if s % every == 0:
            rho, V, v2, P, a2 = ro.primitives(U, prob.gamma)
            q = (P if field == "P" else rho).numpy()
            ts.append(t)
            ph.append(_mode1_phase(q - q.mean()))
        if s == nsteps:
            break
        dt = ro.cfl_dt(U, prob)
        U = ro.ssp_rk2_step(U, dt, prob)
        t += dt
    ph = np.unwrap(np.array(ph))
    slope = np.polyfit(np.array(ts), ph, 1)[0]
    return -slope / (2 * math.pi)            # mode 1 of q(x - c t) has phase -2 pi c t


@pytest.mark.parametrize("var,xi,nsteps", [("pvs", 10.0, 2000), ("pvs", 1.0, 500),
                                            ("dvs", 10.0, 500), ("pms", 10.0, 500)])
def test_sound_wave_speed_is_a_over_xi(var, xi, nsteps):
    w = inputs.sound_wave_1d(256, xi=xi, variant=var)
    c = _phase_speed(w, var, nsteps, 50, "P")
    assert c == pytest.approx(1.0 / xi, rel=0.01)      # a = 1 in this workload


@pytest.mark.parametrize("var,xi", [("pvs", 10.0), ("pms", 10.0), ("pd", 10.0), ("dvs", 1.0)])
def test_entropy_wave_keeps_flow_speed(var, xi):
    w = inputs.contact_1d(256, xi=xi, variant=var)
    u = _phase_speed(w, var, 1000, 100, "rho")
    assert u == pytest.approx(0.01, rel=0.02)


@pytest.mark.parametrize("var,xi", [("pvs", 10.0), ("pms", 10.0), ("pd", 10.0), ("euler", 1.0), ("dvs", 1.0)])
def test_contact_keeps_pressure_and_velocity_uniform(var, xi):
    """Exactly, dP = 0 through MC reconstruction, LLF and the correction.
    Round-off at the unresolved ratio-10 jump seeds a bounded oscillation
    (it grows for ~100 steps and saturates near 1e-5 at xi = 10), so the
    round-off claim is checked over 10 steps (200 at xi = 1)."""
    w = inputs.contact_1d(256, xi=xi, variant=var)
    prob, U = problem_from(w)
    U = ro.run(U, prob, 10 if xi > 1 else 200)
    rho, V, v2, P, a2 = ro.primitives(U, G)
    assert float((P - 1.0 / G).abs().max()) < 1e-13
    assert float((V[0] - 0.01).abs().max()) < 1e-13


@pytest.mark.parametrize("var", ["dvs", "dms"])
def test_density_reduced_forms_create_spurious_pressure(var):
    """Eq. dvs_pr with div V = 0 and grad P = 0: dP/dt = (1 - 1/xi^2) a^2 V.grad(rho).
    Discretely dP/dt = -(1 - 1/xi^2) a^2 drho, drho the Euler mass tendency."""
    xi = 10.0
    w = inputs.contact_1d(256, xi=xi, variant=var)
    prob, U = problem_from(w)
    dU_euler = ro.euler_tendency(U, prob)
    rate = ro.pressure_tendency(U, ro.rhs(U, prob), G)
    rho, V, v2, P, a2 = ro.primitives(U, G)
    want = -(1 - 1 / xi ** 2) * a2 * dU_euler[0]
    assert float(want.abs().max()) > 1e-3
    assert torch.allclose(rate, want, rtol=1e-11, atol=1e-13)
    # at this density ratio the spurious pressure change exceeds P within
    # one step: the density-reduced forms cannot run this flow (Sec. 2.2)
    with pytest.raises(FloatingPointError):
        ro.run(U, prob, 5)
    # a 1% density step only makes the pressure visibly non-uniform
    w = inputs.contact_1d(256, xi=xi, variant=var, ratio=1.01)
    prob, U = problem_from(w)
    U = ro.run(U, prob, 100)
    rho, V, v2, P, a2 = ro.primitives(U, G)
    assert float((P - 1.0 / G).abs().max()) > 1e-6
