"""General equation of state (Sec. 3.2: the reduced equations and the
pressure tendency, Eqs. pvs_cons_dpr / pvs_cons_therm, are stated for any EOS).
The paper specifies no non-ideal gas with parameters; the covolume
(Noble-Abel) gas of oracle/eos.py (also selectable on the float64 device
path through rsst_config.covolume) exercises the general formulas, P = (gamma - 1) e / (1 - b rho), a^2 = gamma P / (rho (1 - b rho)),
(de/dP)_rho = (1 - b rho)/(gamma - 1), (de/drho)_P = -b P/(gamma - 1), to pin
the general formulas: the pressure tendency equals the chain rule of P(U), the
P-forms reduce dP/dt by xi^2, the entropy tendency is unchanged (except PD),
and the characteristic speeds keep the closed forms with this a^2."""
import math

import numpy as np
import pytest
import torch

from oracle import rsst_oracle as ro
from oracle.eos import NobleAbel
from oracle.workload import problem_from
from paper_1812_04135_gb300 import inputs

G = 1.4


EOS = NobleAbel(G, 0.15)


def _states(n, ndim, seed):
    r = inputs.uniform01(seed, (ndim + 2) * n).reshape(ndim + 2, n)
    rho = 0.5 + 2.0 * r[0]
    vel = [0.6 * (2.0 * r[1 + d] - 1.0) for d in range(ndim)]
    p = 0.3 + 1.5 * r[-1]
    v2 = sum(v * v for v in vel)
    eint = EOS.internal_energy(rho, p)
    U = np.stack([rho] + [rho * v for v in vel] + [eint + 0.5 * rho * v2])
    dU = inputs.uniform_pm1(seed + 7, (ndim + 2) * n).reshape(ndim + 2, n)
    return torch.tensor(U), torch.tensor(dU)


def test_ideal_gas_object_is_the_default_path():
    w = inputs.random_smooth_state(2, (20, 14), xi=5.0)
    prob, U = problem_from(w)
    prob2, _ = problem_from(w)
    prob2.gamma = ro.IdealGas(w["gamma"])
    assert torch.equal(ro.run(U, prob, 3), ro.run(U, prob2, 3))


def test_pressure_tendency_is_the_chain_rule_of_P():
    """dP of Eq. pvs_dt_dpr with Eq. pvs_cons_therm = (dP/dU) . dU, the
    derivative taken by complex step through P(U) = P(rho, E - |m|^2/(2 rho))."""
    U, dU = _states(200, 2, 5)
    h = 1e-30
    Uc = U.to(torch.complex128) + 1j * h * dU
    rho = Uc[0]
    eint = Uc[-1] - 0.5 * (Uc[1] ** 2 + Uc[2] ** 2) / rho
    want = (EOS.pressure(rho, eint).imag / h)
    got = ro.pressure_tendency(U, dU, EOS)
    assert torch.allclose(got, want, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("var", [ro.DVS, ro.PVS, ro.DMS, ro.PMS, ro.PD])
def test_reduction_identities_general_eos(var):
    U, dU = _states(300, 3, 9)
    xi = 6.0
    rho, V, v2, P, a2 = ro.primitives(U, EOS)
    dP = ro.pressure_tendency(U, dU, EOS)
    out = ro.rsst_correct(U, dU, var, EOS, xi)
    dPo = ro.pressure_tendency(U, out, EOS)
    tol = dict(rtol=1e-11, atol=1e-11)
    if var in (ro.PVS, ro.PMS, ro.PD):
        assert torch.allclose(dPo, dP / xi ** 2, **tol)
    else:
        assert torch.allclose(out[0], dU[0] / xi ** 2, **tol)
    if var != ro.PD:       # entropy: P_S dS/dt = dP/dt - a^2 drho/dt unchanged
        assert torch.allclose(dPo - a2 * out[0], dP - a2 * dU[0], **tol)


@pytest.mark.parametrize("var", [ro.DVS, ro.PVS, ro.PMS])
def test_characteristic_speeds_general_eos(var):
    rho, u, p, xi = 1.3, 0.37, 0.8, 4.0
    eint = EOS.internal_energy(rho, p)
    U = torch.tensor([rho, rho * u, eint + 0.5 * rho * u * u], dtype=torch.float64)
    a2 = EOS.sound2(rho, p)
    J = np.zeros((3, 3))
    h = 1e-30
    for j in range(3):
        Uc = U.to(torch.complex128).clone()
        Uc[j] += 1j * h
        J[:, j] = (ro.physical_flux(Uc[:, None], 0, EOS)[:, 0].imag / h).numpy()
    M = np.stack([ro.rsst_correct(U[:, None], torch.eye(3, dtype=torch.float64)[:, j:j + 1], var, EOS, xi)[:, 0].numpy()
                  for j in range(3)], axis=1)
    lam = np.sort(np.linalg.eigvals(M @ J).real)
    if var in (ro.DVS, ro.PVS):
        D = (1 - 1 / xi ** 2) ** 2 * u * u + 4 * a2 / xi ** 2
        want = [u, 0.5 * ((1 + 1 / xi ** 2) * u + math.sqrt(D)), 0.5 * ((1 + 1 / xi ** 2) * u - math.sqrt(D))]
    else:
        D = (1 - 1 / xi ** 2) * u * u + a2 / xi ** 2
        want = [u, u + math.sqrt(D), u - math.sqrt(D)]
    assert np.allclose(lam, np.sort(want), rtol=1e-10, atol=1e-12)
