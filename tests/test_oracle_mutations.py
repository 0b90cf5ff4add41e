"""The oracle's pins are sensitive: each plausible mistake below (a wrong
limiter, a min for a max, a dropped term, a flipped sign, an index off by
one, a transposed operand, a first-order time step) is planted in the oracle
on the CPU, one at a time, and at least one of the pins it names must fail.
The mistakes are monkeypatched into the oracle module for the duration of one
test; nothing here touches the CUDA path."""
import math

import pytest
import torch

from oracle import rsst_oracle as ro
from tests import test_oracle_eos as t_eos
from tests import test_oracle_helpers as t_help
from tests import test_oracle_pointwise as t_pt
from tests import test_oracle_time as t_time

ORIG = {name: getattr(ro, name) for name in ("mc_limiter", "llf_flux", "c_tot", "physical_flux", "rsst_correct",
                                              "pressure_tendency", "gravity_source", "ssp_rk2_step", "pad_axis",
                                              "euler_tendency", "cfl_dt", "primitives", "correction_vector")}


# ---- the planted mistakes ----------------------------------------------------

def minmod(a, b):
    return torch.where(a * b > 0, torch.sign(a) * torch.minimum(a.abs(), b.abs()), torch.zeros_like(a))


def central_unlimited(a, b):
    return torch.where(a * b > 0, 0.5 * (a + b), torch.zeros_like(a))


def llf_min_speed(UL, UR, d, gamma, xi, cmax=None):
    cl, cr = ro.c_tot(UL, gamma, xi, cmax), ro.c_tot(UR, gamma, xi, cmax)
    alpha = torch.minimum(cl, cr)
    return 0.5 * (ro.physical_flux(UL, d, gamma) + ro.physical_flux(UR, d, gamma)) - 0.5 * alpha * (UR - UL)


def c_tot_unreduced(U, gamma, xi, cmax=None):
    return ORIG["c_tot"](U, gamma, 1.0, cmax)


def flux_without_pressure_in_momentum(U, d, gamma):
    F = ORIG["physical_flux"](U, d, gamma)
    P = ro.primitives(U, gamma)[3]
    F[1 + d] = F[1 + d] - P
    return F


def flux_energy_without_pressure(U, d, gamma):
    F = ORIG["physical_flux"](U, d, gamma)
    rho, V, v2, P, a2 = ro.primitives(U, gamma)
    F[-1] = U[-1] * V[d]
    return F


def correction_sign_flipped(U, dU, variant, gamma, xi, cmax=None):
    return 2.0 * dU - ORIG["rsst_correct"](U, dU, variant, gamma, xi, cmax)


def correction_f_with_xi_not_xi2(U, dU, variant, gamma, xi, cmax=None):
    # f = 1 - 1/xi instead of 1 - 1/xi^2: the same correction with xi -> sqrt(xi)
    return ORIG["rsst_correct"](U, dU, variant, gamma, math.sqrt(float(xi)), cmax)


def pressure_tendency_vdm_sign(U, dU, gamma):
    eos = ro.as_eos(gamma)
    nd = U.shape[0] - 2
    rho, V, v2, P, a2 = ro.primitives(U, eos)
    vdm = sum(V[e] * dU[1 + e] for e in range(nd))
    return ORIG["pressure_tendency"](U, dU, gamma) + 2.0 * vdm / eos.de_dP(rho, P)


def pvs_energy_row_with_minus_kinetic(U, variant, gamma):
    which, r = ORIG["correction_vector"](U, variant, gamma)
    if variant == ro.PVS:
        rho, V, v2, P, a2 = ro.primitives(U, gamma)
        r = list(r)
        r[-1] = r[-1] - v2 / a2  # (e + P + rho V^2/2) -> (e + P - rho V^2/2) in the PVS energy row
    return which, r


def gravity_without_energy_work(U, prob):
    G = ORIG["gravity_source"](U, prob)
    G[-1] = torch.zeros_like(G[-1])
    return G


def forward_euler(U, dt, prob):
    return U + dt * ro.rhs(U, prob)


def rk2_second_stage_at_the_old_state(U, dt, prob):
    Us = U + dt * ro.rhs(U, prob)
    return 0.5 * U + 0.5 * (Us + dt * ro.rhs(U, prob))


def wall_without_sign_flip(U, d, prob):
    ax = prob.axis(d)
    n = U.shape[ax]
    if prob.bc[d] == ro.PERIODIC:
        return ORIG["pad_axis"](U, d, prob)
    return torch.cat([torch.flip(U.narrow(ax, 0, 2), dims=[ax]), U, torch.flip(U.narrow(ax, n - 2, 2), dims=[ax])], dim=ax)


def wall_ghost_off_by_one(U, d, prob):
    ax = prob.axis(d)
    n = U.shape[ax]
    if prob.bc[d] == ro.PERIODIC:
        return ORIG["pad_axis"](U, d, prob)
    P = ORIG["pad_axis"](U, d, prob)
    # ghost -1 takes the image of interior cell 1 instead of 0
    lo = P.narrow(ax, 0, 2).clone()
    lo.narrow(ax, 1, 1).copy_(P.narrow(ax, 0, 1))
    return torch.cat([lo, P.narrow(ax, 2, n + 2)], dim=ax)


def divergence_with_the_other_width(U, prob):
    dU = torch.zeros_like(U)
    for d in range(prob.ndim):
        ax = prob.axis(d)
        F = ro.face_fluxes(U, d, prob)
        n = U.shape[ax]
        dU = dU - (F.narrow(ax, 1, n) - F.narrow(ax, 0, n)) / prob.dx[prob.ndim - 1 - d]
    return dU


def cfl_max_instead_of_sum(U, prob):
    with torch.no_grad():
        c = ro.c_tot(U, prob.gamma, float(prob.xi), prob.cmax)
        rate = torch.stack([c / prob.dx[d] for d in range(prob.ndim)]).amax(dim=0)
        return float(prob.cfl / rate.max())


def pressure_without_kinetic_energy(U, gamma):
    rho, V, v2, P, a2 = ORIG["primitives"](U, gamma)
    eos = ro.as_eos(gamma)
    P = eos.pressure(rho, U[-1])
    return rho, V, v2, P, eos.sound2(rho, P)


# ---- which pins must catch each -----------------------------------------------

MUTATIONS = {
    "MC replaced by minmod": ("mc_limiter", minmod, [t_pt.test_mc_limiter_hand_cases]),
    "MC without the 2a, 2b bounds": ("mc_limiter", central_unlimited, [t_pt.test_mc_limiter_hand_cases]),
    "LLF speed min instead of max": ("llf_flux", llf_min_speed, [t_pt.test_llf_flux_consistency_and_upwinding]),
    "c_tot without the 1/xi": ("c_tot", c_tot_unreduced,
                               [lambda: t_time.test_cfl_is_the_acoustic_courant_condition_at_rest((16,), (0.1,), 7.0)]),
    "momentum flux without P": ("physical_flux", flux_without_pressure_in_momentum,
                                [lambda: t_help.test_face_flux_of_a_uniform_state_is_the_euler_flux(0)]),
    "energy flux E V instead of (E + P) V": ("physical_flux", flux_energy_without_pressure,
                                             [lambda: t_help.test_face_flux_of_a_uniform_state_is_the_euler_flux(1)]),
    "RSST correction added instead of subtracted": ("rsst_correct", correction_sign_flipped,
                                                    [lambda: t_pt.test_pointwise_identities(1)]),
    "f = 1 - 1/xi instead of 1 - 1/xi^2": ("rsst_correct", correction_f_with_xi_not_xi2,
                                           [lambda: t_pt.test_pointwise_identities(1)]),
    "pressure tendency with +V.dm": ("pressure_tendency", pressure_tendency_vdm_sign,
                                     [t_eos.test_pressure_tendency_is_the_chain_rule_of_P,
                                      lambda: t_pt.test_pointwise_identities(2)]),
    "PVS energy row with -rho V^2/2": ("correction_vector", pvs_energy_row_with_minus_kinetic,
                                       [lambda: t_pt.test_pointwise_identities(2)]),
    "gravity without the work term m.F": ("gravity_source", gravity_without_energy_work,
                                          [t_pt.test_gravity_leaves_pressure_tendency_unchanged]),
    "forward Euler instead of SSP-RK2": ("ssp_rk2_step", forward_euler,
                                         [lambda: t_time.test_entropy_wave_converges_at_second_order(ro.EULER, 1.0)]),
    "RK2 second stage evaluated at U^n": ("ssp_rk2_step", rk2_second_stage_at_the_old_state,
                                          [lambda: t_time.test_entropy_wave_converges_at_second_order(ro.EULER, 1.0)]),
    "wall without the normal-momentum sign": ("pad_axis", wall_without_sign_flip,
                                              [lambda: t_help.test_reflecting_ghosts_mirror_with_normal_momentum_negated(0)]),
    "wall ghost -1 mirrors cell 1": ("pad_axis", wall_ghost_off_by_one,
                                     [lambda: t_help.test_reflecting_ghosts_mirror_with_normal_momentum_negated(1)]),
    "divergence divided by the other axis' width": ("euler_tendency", divergence_with_the_other_width,
                                                    [lambda: t_time.test_entropy_wave_on_an_anisotropic_grid(ro.EULER, 1.0)]),
    "CFL rate max over axes instead of sum": ("cfl_dt", cfl_max_instead_of_sum,
                                              [lambda: t_time.test_cfl_is_the_acoustic_courant_condition_at_rest(
                                                  (8, 6), (0.1, 0.03), 1.0)]),
    "pressure without the kinetic energy": ("primitives", pressure_without_kinetic_energy,
                                            [lambda: t_help.test_face_flux_of_a_uniform_state_is_the_euler_flux(0)]),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_fails_a_pin(name, monkeypatch):
    attr, bad, pins = MUTATIONS[name]
    for pin in pins:                       # the pins pass on the real oracle
        pin()
    monkeypatch.setattr(ro, attr, bad)
    caught = []
    for pin in pins:
        try:
            pin()
        except (AssertionError, FloatingPointError, pytest.fail.Exception) as e:
            caught.append(type(e).__name__)
    assert caught, f"no pin caught: {name}"
