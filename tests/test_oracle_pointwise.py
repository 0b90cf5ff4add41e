"""Oracle pins that need no time integration: limiter and flux hand cases,
the pointwise RSST identities (Sec. 3.2, App. A), the characteristic speeds
of the linearised reduced system (Eqs. dvs_lambda1/2, pms_speed), xi = 1
reducing to the Euler step (Sec. 3.2) and exact steadiness of a uniform state
(Sec. 3.2, steady solutions unchanged)."""
import math

import numpy as np
import pytest
import torch

from oracle import rsst_oracle as ro
from oracle.workload import problem_from
from paper_1812_04135_gb300 import inputs

G = 5.0 / 3.0


def test_mc_limiter_hand_cases():
    a = torch.tensor([1.0, 1.0, 1.0, -2.0, 0.0, 3.0, 1.0, -1.0], dtype=torch.float64)
    b = torch.tensor([1.0, 3.0, 0.2, -1.0, 5.0, -1.0, 10.0, -0.25], dtype=torch.float64)
    # (a+b)/2 when a~b; 2b when b much smaller; 2a when a much smaller; 0 on sign change
    want = [1.0, 2.0, 0.4, -1.5, 0.0, 0.0, 2.0, -0.5]
    assert ro.mc_limiter(a, b).tolist() == want
    # odd and positively homogeneous
    x = torch.randn(1000, dtype=torch.float64)
    y = torch.randn(1000, dtype=torch.float64)
    assert torch.equal(ro.mc_limiter(-x, -y), -ro.mc_limiter(x, y))
    assert torch.allclose(ro.mc_limiter(3 * x, 3 * y), 3 * ro.mc_limiter(x, y), rtol=1e-15, atol=0)


def test_llf_flux_consistency_and_upwinding():
    # consistency: F_hat(U, U) = F(U)
    U = torch.tensor([[1.2], [0.3], [-0.1], [2.5]], dtype=torch.float64)
    for d in range(2):
        assert torch.equal(ro.llf_flux(U, U, d, G, 3.0), ro.physical_flux(U, d, G))
    # hand value: 1D, rho=1, u=0, P=1 on both sides except rho_R = 2 (same P)
    UL = torch.tensor([[1.0], [0.0], [1.0 / (G - 1)]], dtype=torch.float64)
    UR = torch.tensor([[2.0], [0.0], [1.0 / (G - 1)]], dtype=torch.float64)
    xi = 4.0
    alpha = max(math.sqrt(G * 1.0 / 1.0), math.sqrt(G * 1.0 / 2.0)) / xi
    F = ro.llf_flux(UL, UR, 0, G, xi)[:, 0].tolist()
    assert F[0] == pytest.approx(-0.5 * alpha * 1.0, rel=1e-15)
    assert F[1] == pytest.approx(1.0, rel=1e-15)
    assert F[2] == pytest.approx(0.0, abs=1e-15)


def _random_states(n, ndim, seed):
    r = inputs.uniform01(seed, (ndim + 2) * n).reshape(ndim + 2, n)
    rho = 0.5 + 2.0 * r[0]
    vel = [0.6 * (2.0 * r[1 + d] - 1.0) for d in range(ndim)]
    p = 0.3 + 1.5 * r[-1]
    v2 = sum(v * v for v in vel)
    U = np.stack([rho] + [rho * v for v in vel] + [p / (G - 1) + 0.5 * rho * v2])
    dU = inputs.uniform_pm1(seed + 7, (ndim + 2) * n).reshape(ndim + 2, n)
    return torch.tensor(U), torch.tensor(dU)


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_pointwise_identities(ndim):
    U, dU = _random_states(512, ndim, 3 + ndim)
    xi = 7.0
    rho, V, v2, P, a2 = ro.primitives(U, G)
    dP = ro.pressure_tendency(U, dU, G)
    ent = dP - a2 * dU[0]                         # P_S dS/dt = dP - a^2 drho
    vel = [(dU[1 + d] - V[d] * dU[0]) / rho for d in range(ndim)]
    for var in (ro.DVS, ro.PVS, ro.DMS, ro.PMS, ro.PD):
        out = ro.rsst_correct(U, dU, var, G, xi)
        dPo = ro.pressure_tendency(U, out, G)
        tol = dict(rtol=1e-12, atol=1e-12)
        if var in (ro.PVS, ro.PMS, ro.PD):       # dP/dt = dP / xi^2 (Eq. pvs_prim, pms_prim, pd_prim)
            assert torch.allclose(dPo, dP / xi ** 2, **tol)
        if var in (ro.DVS, ro.DMS):               # drho/dt = drho / xi^2 (Eq. dvs_prim, dms_prim)
            assert torch.allclose(out[0], dU[0] / xi ** 2, **tol)
        if var != ro.PD:                          # entropy equation unchanged (Sec. 3.2)
            assert torch.allclose(dPo - a2 * out[0], ent, **tol)
        else:                                     # Eq. pd_entropy: P_S DS/Dt changes by -(1-1/xi^2) dP
            f = 1 - 1 / xi ** 2
            assert torch.allclose(dPo - a2 * out[0], ent - f * dP, **tol)
        if var in (ro.PVS, ro.DVS, ro.PD):        # velocity equation unchanged
            for d in range(ndim):
                assert torch.allclose((out[1 + d] - V[d] * out[0]) / rho, vel[d], **tol)
        if var in (ro.PMS, ro.DMS, ro.PD):        # momentum equation unchanged
            assert torch.equal(out[1:1 + ndim], dU[1:1 + ndim])
        if var == ro.PD:                          # mass equation unchanged
            assert torch.equal(out[0], dU[0])


def _flux_jacobian(U, gamma):
    """Exact Jacobian dF_x/dU of the 1D Euler flux by complex-step differentiation."""
    n = U.shape[0]
    J = np.zeros((n, n))
    h = 1e-30
    for j in range(n):
        Uc = U.to(torch.complex128).clone()
        Uc[j] += 1j * h
        J[:, j] = (ro.physical_flux(Uc[:, None], 0, gamma)[:, 0].imag / h).numpy()
    return J


@pytest.mark.parametrize("var", [ro.DVS, ro.PVS, ro.DMS, ro.PMS, ro.PD])
@pytest.mark.parametrize("xi", [1.0, 3.0, 25.0])
def test_characteristic_speeds(var, xi):
    """Eigenvalues of (I - f r l^T) dF/dU in conservative variables equal the
    wave speeds of the primitive reduced systems."""
    rho, u, p = 1.3, 0.37, 0.8
    U = torch.tensor([rho, rho * u, p / (G - 1) + 0.5 * rho * u * u], dtype=torch.float64)
    a2 = G * p / rho
    J = _flux_jacobian(U, G)
    M = np.zeros((3, 3))
    for j in range(3):
        e = torch.zeros(3, 1, dtype=torch.float64)
        e[j, 0] = 1.0
        M[:, j] = ro.rsst_correct(U[:, None], e, var, G, xi)[:, 0].numpy()
    lam = np.sort(np.linalg.eigvals(M @ J).real)
    if var in (ro.DVS, ro.PVS, ro.PD):            # Eqs. dvs_lambda1, dvs_lambda2
        D = (1 - 1 / xi ** 2) ** 2 * u * u + 4 * a2 / xi ** 2
        want = [u, 0.5 * ((1 + 1 / xi ** 2) * u + math.sqrt(D)), 0.5 * ((1 + 1 / xi ** 2) * u - math.sqrt(D))]
    else:                                         # Eq. pms_speed
        D = (1 - 1 / xi ** 2) * u * u + a2 / xi ** 2
        want = [u, u + math.sqrt(D), u - math.sqrt(D)]
    assert np.allclose(lam, np.sort(want), rtol=1e-10, atol=1e-12)


def test_low_mach_sound_speed_limit():
    """At V = 0 every form has sound speeds +-a/xi (Sec. 2.1, App. A.2)."""
    U = torch.tensor([1.0, 0.0, 1.0 / (G - 1)], dtype=torch.float64)
    J = _flux_jacobian(U, G)
    for var in (ro.DVS, ro.PVS, ro.DMS, ro.PMS, ro.PD):
        M = np.stack([ro.rsst_correct(U[:, None], torch.eye(3, dtype=torch.float64)[:, j:j + 1], var, G, 10.0)[:, 0].numpy()
                      for j in range(3)], axis=1)
        lam = np.sort(np.linalg.eigvals(M @ J).real)
        assert np.allclose(lam, [-math.sqrt(G) / 10, 0.0, math.sqrt(G) / 10], atol=1e-13)


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_xi_one_is_euler_bitwise(ndim):
    n = {1: (40,), 2: (20, 12), 3: (10, 8, 6)}[ndim]
    w = inputs.random_smooth_state(ndim, n, xi=1.0)
    prob, U = problem_from(w)
    ref = ro.run(U, problem_from(w, variant="euler")[0], 3)
    for var in ("dvs", "pvs", "dms", "pms", "pd"):
        got = ro.run(U, problem_from(w, variant=var)[0], 3)
        assert torch.equal(got, ref), var


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_uniform_state_is_steady(ndim):
    n = {1: (16,), 2: (8, 6), 3: (6, 4, 5)}[ndim]
    w = inputs.uniform_state(ndim, n)
    for var in ("euler", "dvs", "pvs", "dms", "pms", "pd"):
        prob, U = problem_from(w, variant=var)
        assert torch.equal(ro.run(U, prob, 2), U)


def test_gravity_leaves_pressure_tendency_unchanged():
    """App. B: the force terms (0, rho F, m.F) carry no pressure tendency."""
    U, _ = _random_states(256, 3, 21)
    w = inputs.uniform_state(3, (4, 4, 4))
    prob, _ = problem_from(w)
    prob.grav = (0.3, -1.2, 0.7)
    src = ro.gravity_source(U, prob)
    assert torch.allclose(ro.pressure_tendency(U, src, G), torch.zeros(256, dtype=torch.float64), atol=1e-14)
