"""Pins of the oracle's helpers that the step-level pins reach only
indirectly: the ghost cells of each boundary (reading 7), the consistency of
the face fluxes (Sec. 4.2: the LLF flux of a uniform state is its Euler
flux), the kinetic-energy functional the adjoint differentiates (closed-form
values) and its gradient, and
the non-physical check (reading 9).  Expected values are written out index by
index in Python, not with the tensor operations the oracle uses."""
import math

import pytest
import torch

from oracle import rsst_oracle as ro

DT = torch.float64


def prob2d(n, bc, **kw):
    return ro.Problem(ndim=2, n=n, dx=(0.1, 0.2), gamma=1.4, bc=bc, **kw)


def random_state(n, seed=0):
    g = torch.Generator().manual_seed(seed)
    ny, nx = n[1], n[0]
    rho = 1.0 + torch.rand(ny, nx, generator=g, dtype=DT)
    mx, my = torch.rand(ny, nx, generator=g, dtype=DT) - 0.5, torch.rand(ny, nx, generator=g, dtype=DT) - 0.5
    E = 3.0 + torch.rand(ny, nx, generator=g, dtype=DT)
    return torch.stack([rho, mx, my, E])


@pytest.mark.parametrize("d", [0, 1])
def test_periodic_ghosts_wrap(d):
    n = (5, 4)
    prob = prob2d(n, (ro.PERIODIC, ro.PERIODIC))
    U = random_state(n)
    P = ro.pad_axis(U, d, prob)
    nd = n[d]
    for v in range(4):
        for j in range(P.shape[1]):
            for i in range(P.shape[2]):
                k = (i if d == 0 else j) - 2          # interior index along d (ghosts: -2, -1, nd, nd+1)
                src = k % nd
                jj, ii = (j, src) if d == 0 else (src, i)
                assert P[v, j, i] == U[v, jj, ii]


@pytest.mark.parametrize("d", [0, 1])
def test_reflecting_ghosts_mirror_with_normal_momentum_negated(d):
    n = (5, 4)
    prob = prob2d(n, (ro.REFLECT, ro.REFLECT))
    U = random_state(n, seed=1)
    P = ro.pad_axis(U, d, prob)
    nd = n[d]
    for v in range(4):
        sign = -1.0 if v == 1 + d else 1.0
        for j in range(P.shape[1]):
            for i in range(P.shape[2]):
                k = (i if d == 0 else j) - 2
                if 0 <= k < nd:
                    src, s = k, 1.0
                elif k < 0:
                    src, s = -1 - k, sign                 # ghost -1 mirrors 0, ghost -2 mirrors 1
                else:
                    src, s = 2 * nd - 1 - k, sign         # ghost n mirrors n-1, ghost n+1 mirrors n-2
                jj, ii = (j, src) if d == 0 else (src, i)
                assert P[v, j, i] == s * U[v, jj, ii]


def test_wall_ghosts_of_the_background_are_the_background():
    """A state equal to its hydrostatic background (at rest) gets the
    background's own ghost values at the walls: ghost = U0(ghost) +
    mirror(U - U0) with U - U0 = 0."""
    n = (3, 6)
    gamma = 1.4
    z = [(k - 2 + 0.5) / 6 for k in range(10)]
    rho0 = torch.tensor([math.exp(-zz) for zz in z], dtype=DT)
    p0 = torch.tensor([math.exp(-zz) / gamma for zz in z], dtype=DT)
    prob = prob2d(n, (ro.PERIODIC, ro.REFLECT), vertical=1, bg_rho=rho0, bg_p=p0)
    U = torch.zeros(4, 6, 3, dtype=DT)
    for j in range(6):
        U[0, j, :] = rho0[j + 2]
        U[3, j, :] = p0[j + 2] / (gamma - 1.0)
    P = ro.pad_axis(U, 1, prob)
    for k in range(10):
        for i in range(3):
            assert P[0, k, i] == pytest.approx(float(rho0[k]), rel=1e-15, abs=0)
            assert P[1, k, i] == 0.0 and P[2, k, i] == 0.0
            assert P[3, k, i] == pytest.approx(float(p0[k]) / (gamma - 1.0), rel=1e-15, abs=0)


@pytest.mark.parametrize("d", [0, 1])
def test_face_flux_of_a_uniform_state_is_the_euler_flux(d):
    """Consistency of the LLF flux: with U_L = U_R = U the dissipation term
    vanishes and the face flux is F(U) = (m_d, m V_d + P e_d, (E + P) V_d)."""
    n = (4, 3)
    rho, vx, vy, p, gamma = 1.3, 0.4, -0.7, 0.9, 1.4
    prob = ro.Problem(ndim=2, n=n, dx=(0.1, 0.2), gamma=gamma, xi=5.0)
    E = p / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy)
    U = torch.stack([torch.full((3, 4), c, dtype=DT) for c in (rho, rho * vx, rho * vy, E)])
    Fh = ro.face_fluxes(U, d, prob)
    vd = (vx, vy)[d]
    want = [rho * vd, rho * vx * vd + (p if d == 0 else 0.0), rho * vy * vd + (p if d == 1 else 0.0), (E + p) * vd]
    for v in range(4):
        assert torch.allclose(Fh[v], torch.full_like(Fh[v], want[v]), rtol=1e-15, atol=1e-15)


def test_kinetic_energy_gradient_matches_central_differences():
    n = (4, 3)
    prob = ro.Problem(ndim=2, n=n, dx=(0.1, 0.2), gamma=1.4)
    U = random_state(n, seed=2)
    G = ro.kinetic_energy_gradient(U, prob)
    h = 1e-6
    for v in range(4):
        for j in range(3):
            for i in range(4):
                Up, Um = U.clone(), U.clone()
                Up[v, j, i] += h
                Um[v, j, i] -= h
                fd = (float(ro.kinetic_energy(Up, prob)) - float(ro.kinetic_energy(Um, prob))) / (2 * h)
                assert G[v, j, i] == pytest.approx(fd, rel=1e-7, abs=1e-10)


def _moving_gas(ndim, n, rho, V, E):
    shape = tuple(reversed(n))
    return torch.stack([torch.full(shape, rho, dtype=DT)] + [torch.full(shape, rho * V[d], dtype=DT)
                                                              for d in range(ndim)] + [torch.full(shape, E, dtype=DT)])


@pytest.mark.parametrize("ndim,n,dx", [(1, (10,), (0.3,)), (2, (6, 5), (0.1, 0.4)),
                                       (3, (4, 3, 5), (0.2, 0.5, 0.125))])
def test_kinetic_energy_of_a_uniform_moving_gas(ndim, n, dx):
    """J of a gas moving uniformly is 1/2 rho |V|^2 times the domain volume
    (n_d dx_d along every axis): a dropped 1/2, a missing cell width, or m^2
    instead of m^2/rho (rho != 1 here) changes it."""
    rho, V = 2.5, (0.3, -0.7, 1.1)[:ndim]
    prob = ro.Problem(ndim=ndim, n=n, dx=dx, gamma=1.4)
    volume = 1.0
    for d in range(ndim):
        volume *= n[d] * dx[d]
    want = 0.5 * rho * sum(v * v for v in V) * volume
    assert float(ro.kinetic_energy(_moving_gas(ndim, n, rho, V, 9.0), prob)) == pytest.approx(want, rel=1e-14)


def test_kinetic_energy_of_a_sine_velocity():
    """V_x = sin(2 pi x_i) at the N cell centres of [0, 1), rho = 3: the sum of
    sin^2 over a full period of N >= 3 points is N/2, so J = 1/2 rho (1/2) L
    with L = N dx = 1."""
    N = 16
    x = (torch.arange(N, dtype=DT) + 0.5) / N
    rho = 3.0
    v = torch.sin(2 * math.pi * x)
    U = torch.stack([torch.full((N,), rho, dtype=DT), rho * v, torch.full((N,), 10.0, dtype=DT)])
    prob = ro.Problem(ndim=1, n=(N,), dx=(1.0 / N,), gamma=1.4)
    assert float(ro.kinetic_energy(U, prob)) == pytest.approx(0.5 * rho * 0.5, rel=1e-14)


@pytest.mark.parametrize("field,value", [(0, 0.0), (0, -1.0), (3, 0.1), (1, float("nan")), (3, float("inf"))])
def test_check_physical_rejects_bad_cells(field, value):
    n = (4, 3)
    prob = ro.Problem(ndim=2, n=n, dx=(0.1, 0.2), gamma=1.4)
    U = random_state(n, seed=3)
    ro.check_physical(U, prob)             # a physical state passes
    U[field, 1, 2] = value
    if field == 3 and value == 0.1:
        U[1, 1, 2], U[2, 1, 2] = 2.0, 0.0  # kinetic energy |m|^2/(2 rho) = 2/rho > E = 0.1: P < 0
    with pytest.raises(FloatingPointError):
        ro.check_physical(U, prob)
