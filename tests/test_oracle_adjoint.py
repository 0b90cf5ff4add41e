"""The oracle's discrete adjoint (reverse-mode derivative of its own step)
against central finite differences of the forward oracle and against a
forward-mode directional derivative (dot-product test)."""
import pytest
import torch

from oracle import adjoint as adj
from oracle import rsst_oracle as ro
from oracle.workload import problem_from
from paper_1812_04135_gb300 import inputs


def _case():
    w = inputs.polytrope_2d(12, 16, xi=20.0, contrast=20.0, amp=1e-2)
    prob, U = problem_from(w)
    # give it some motion so the kinetic energy has a non-trivial gradient
    U = ro.run(U, prob, 3)
    dt = ro.cfl_dt(U, prob)
    return prob, U, dt


def _J(U0, prob, nsteps, dt):
    with torch.no_grad():
        U = U0
        for _ in range(nsteps):
            U = ro.ssp_rk2_step(U, dt, prob)
        return float(ro.kinetic_energy(U, prob))


def test_adjoint_matches_central_differences():
    prob, U0, dt = _case()
    nsteps, every = 6, 4
    J, UN, lam, dxi = adj.adjoint_run(U0, prob, nsteps, dt, every)
    assert J == pytest.approx(_J(U0, prob, nsteps, dt), rel=1e-14)
    eps = 1e-6
    idx = [(0, 3, 5), (0, 0, 0), (0, 15, 11), (1, 7, 2), (2, 0, 6), (3, 9, 9)]
    for (c, j, i) in idx:
        h = eps * abs(float(U0[c, j, i])) if c in (0, 3) else 1e-7
        Up = U0.clone(); Up[c, j, i] += h
        Um = U0.clone(); Um[c, j, i] -= h
        fd = (_J(Up, prob, nsteps, dt) - _J(Um, prob, nsteps, dt)) / (2 * h)
        assert float(lam[c, j, i]) == pytest.approx(fd, rel=2e-5, abs=1e-9 * abs(J) / h), (c, j, i)
    hx = 1e-6 * float(prob.xi)
    from dataclasses import replace
    fdx = (_J(U0, replace(prob, xi=float(prob.xi) + hx), nsteps, dt)
           - _J(U0, replace(prob, xi=float(prob.xi) - hx), nsteps, dt)) / (2 * hx)
    assert dxi == pytest.approx(fdx, rel=2e-5)


def test_dot_product_identity():
    prob, U0, dt = _case()
    v = torch.tensor(inputs.uniform_pm1(77, U0.numel()).reshape(U0.shape)) * 1e-3
    lam = torch.tensor(inputs.uniform_pm1(78, U0.numel()).reshape(U0.shape))
    from torch.func import jvp
    _, Jv = jvp(lambda X: ro.ssp_rk2_step(X, dt, prob), (U0,), (v,))
    JTlam, _ = adj.step_vjp(U0, lam, dt, prob)
    lhs = float((lam * Jv).sum())
    rhs = float((JTlam * v).sum())
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_density_gradient_at_fixed_velocity_and_pressure():
    """The chain rule of the conserved-state gradient to a density change at
    fixed V and P, against central differences of J over such changes."""
    prob, U0, dt = _case()
    nsteps, every = 4, 2
    J, UN, lam, dxi = adj.adjoint_run(U0, prob, nsteps, dt, every)
    g = adj.rho_gradient_fixed_vp(U0, lam, prob.gamma)
    rho, V, v2, P, a2 = ro.primitives(U0, prob.gamma)

    def at_rho(j, i, r):
        U = U0.clone()
        vx, vy = float(V[0][j, i]), float(V[1][j, i])
        U[0, j, i] = r
        U[1, j, i] = r * vx
        U[2, j, i] = r * vy
        U[3, j, i] = float(P[j, i]) / (prob.gamma - 1.0) + 0.5 * r * (vx * vx + vy * vy)
        return U

    for (j, i) in [(3, 5), (0, 0), (15, 11), (8, 2)]:
        r0 = float(rho[j, i])
        h = 1e-6 * r0
        fd = (_J(at_rho(j, i, r0 + h), prob, nsteps, dt) - _J(at_rho(j, i, r0 - h), prob, nsteps, dt)) / (2 * h)
        assert float(g[j, i]) == pytest.approx(fd, rel=2e-5, abs=1e-9 * abs(J) / h), (j, i)
    # at V = 0 it is the fixed-(m, E) gradient plus (de/drho)_P lam_E, which is 0 for an ideal gas
    Z = U0.clone()
    Z[1:3] = 0.0
    Z[3] = P / (prob.gamma - 1.0)
    assert torch.equal(adj.rho_gradient_fixed_vp(Z, lam, prob.gamma), lam[0])
