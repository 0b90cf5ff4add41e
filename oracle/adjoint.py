"""Discrete adjoint of the oracle's SSP-RK2 step (TEST INFRASTRUCTURE ONLY).

The discrete adjoint of a step is, by definition, the transpose of the
Jacobian of the discrete map U^n -> U^{n+1}.  Here it is obtained by
reverse-mode differentiation (torch.autograd) of the plain oracle step in
``rsst_oracle``; non-smooth operations take the branch the forward pass took
(MC limiter branch, LLF max with ties to the left state, |V| with a zero
subgradient at V = 0).

Conventions (the paper has no adjoint, so these are this project's
readings): dt is fixed for the whole run and not differentiated; the
functional is the final kinetic energy J = sum |m|^2/(2 rho) dV; gradients are
taken with respect to every component of the initial conserved state (the
density gradient at fixed m and E is component 0) and with respect to xi.

Pinned in tests/test_oracle_adjoint.py by central finite differences of the
forward oracle and by a dot-product (transpose) identity against a
forward-mode directional derivative.
"""
from __future__ import annotations

from dataclasses import replace
from typing import Callable, Optional

import torch

from . import rsst_oracle as ro


def step_vjp(U: torch.Tensor, lam: torch.Tensor, dt: float, prob: ro.Problem):
    """Return (lambda^T dU^{n+1}/dU^n, lambda^T dU^{n+1}/dxi) for one step from U."""
    Uc = U.detach().clone().requires_grad_(True)
    xi_t = torch.tensor(float(prob.xi), dtype=ro.DT, requires_grad=True)
    out = ro.ssp_rk2_step(Uc, dt, replace(prob, xi=xi_t))
    gU, gxi = torch.autograd.grad(out, [Uc, xi_t], grad_outputs=lam, allow_unused=True)
    return gU, 0.0 if gxi is None else float(gxi)


def stage_vjp(U: torch.Tensor, lam: torch.Tensor, prob: ro.Problem):
    """Return (lambda^T dL/dU, lambda^T dL/dxi) of the right-hand side L at U."""
    Uc = U.detach().clone().requires_grad_(True)
    xi_t = torch.tensor(float(prob.xi), dtype=ro.DT, requires_grad=True)
    out = ro.rhs(Uc, replace(prob, xi=xi_t))
    gU, gxi = torch.autograd.grad(out, [Uc, xi_t], grad_outputs=lam, allow_unused=True)
    return gU, 0.0 if gxi is None else float(gxi)


def adjoint_run(U0: torch.Tensor, prob: ro.Problem, nsteps: int, dt: float, every: int,
                lam_final: Optional[Callable] = None):
    """Forward nsteps from U0 with checkpoints every ``every`` steps, then the
    reverse sweep segment by segment with recomputation.

    Returns (J, U_final, dJ/dU0, dJ/dxi) for J = kinetic energy of U_final
    (or, when ``lam_final`` is given, dJ/dU_final = lam_final(U_final)).
    """
    xi0 = float(prob.xi)
    pf = replace(prob, xi=xi0)
    ckpts = []
    U = U0.detach().clone()
    with torch.no_grad():
        for s in range(nsteps):
            if s % every == 0:
                ckpts.append(U.clone())
            U = ro.ssp_rk2_step(U, dt, pf)
    J = float(ro.kinetic_energy(U, pf))
    lam = (lam_final or (lambda X: ro.kinetic_energy_gradient(X, pf)))(U)
    dxi = 0.0
    for seg in reversed(range(len(ckpts))):
        s0 = seg * every
        s1 = min(s0 + every, nsteps)
        Uc = ckpts[seg].clone().requires_grad_(True)
        xi_t = torch.tensor(xi0, dtype=ro.DT, requires_grad=True)
        p = replace(prob, xi=xi_t)
        Ue = Uc
        for _ in range(s0, s1):
            Ue = ro.ssp_rk2_step(Ue, dt, p)
        gU, gxi = torch.autograd.grad(Ue, [Uc, xi_t], grad_outputs=lam, allow_unused=True)
        lam = gU.detach()
        dxi += 0.0 if gxi is None else float(gxi)
    return J, U, lam, dxi


def rho_gradient_fixed_vp(U0: torch.Tensor, lam0: torch.Tensor, gamma) -> torch.Tensor:
    """Density gradient at fixed velocity and pressure from the conserved-state
    gradient (the optional chain rule of the adjoint readings): with
    m = rho V and E = e(rho, P) + rho |V|^2/2,
    dJ/drho|_{V,P} = lam_rho + V . lam_m + [(de/drho)_P + |V|^2/2] lam_E."""
    eos = ro.as_eos(gamma)
    rho, V, v2, P, a2 = ro.primitives(U0, eos)
    nd = U0.shape[0] - 2
    out = lam0[0] + (eos.de_drho(rho, P) + 0.5 * v2) * lam0[-1]
    for d in range(nd):
        out = out + V[d] * lam0[1 + d]
    return out
