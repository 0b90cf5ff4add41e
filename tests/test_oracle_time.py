"""Pins of the oracle's time step: the CFL rule (reading: dt = C / max over
cells of sum_d c_tot / dx_d, C = 0.4, Sec. 4.2) and the SSP-RK2 stage
combination (Sec. 4.2, Gottlieb et al.), against what the mathematics fixes:

* on a uniform gas at rest c_tot = a/xi, so the rule is the textbook acoustic
  Courant condition (a/xi) dt sum_d 1/dx_d = C;
* dt is invariant in form under the scalings of the Euler equations: all
  speeds times k (m -> k m, E -> k^2 E) gives dt / k, all lengths times k
  gives k dt;
* a smooth entropy wave advected once around a periodic domain converges at
  second order in space and time together (a first-order or unstable time
  combination fails this).
"""
import math

import pytest
import torch

from oracle import rsst_oracle as ro

DT = torch.float64


def problem(n, dx, xi=1.0, variant=ro.EULER, gamma=1.4, cfl_rule=0):
    nd = len(n)
    return ro.Problem(ndim=nd, n=tuple(n), dx=tuple(dx), gamma=gamma, xi=xi, variant=variant, grav=(0.0, 0.0, 0.0),
                      bc=(ro.PERIODIC,) * nd, cfl=0.4, vertical=-1, bg_rho=None, bg_p=None, cmax=None,
                      cfl_rule=cfl_rule)


def uniform(n, rho, vel, p, gamma=1.4):
    shape = tuple(reversed(n))
    comps = [torch.full(shape, rho, dtype=DT)]
    comps += [torch.full(shape, rho * v, dtype=DT) for v in vel]
    comps.append(torch.full(shape, p / (gamma - 1) + 0.5 * rho * sum(v * v for v in vel), dtype=DT))
    return torch.stack(comps)


@pytest.mark.parametrize("n,dx", [((16,), (0.1,)), ((8, 6), (0.1, 0.03)), ((4, 5, 6), (0.2, 0.05, 0.01))])
@pytest.mark.parametrize("xi", [1.0, 7.0])
def test_cfl_is_the_acoustic_courant_condition_at_rest(n, dx, xi):
    gamma, rho, p = 1.4, 1.7, 0.9
    U = uniform(n, rho, (0.0,) * len(n), p, gamma)
    dt = ro.cfl_dt(U, problem(n, dx, xi=xi, gamma=gamma))
    a = math.sqrt(gamma * p / rho)
    courant = (a / xi) * dt * sum(1.0 / h for h in dx)
    assert courant == pytest.approx(0.4, rel=1e-13)


@pytest.mark.parametrize("n,dx", [((16,), (0.1,)), ((8, 6), (0.1, 0.03)), ((4, 5, 6), (0.2, 0.05, 0.01))])
def test_min_width_cfl_rule_at_rest(n, dx):
    """The other reading of the multi-dimensional CFL step: (a/xi) dt / min dx = C;
    in 1D it is the same step as the sum rule."""
    gamma, rho, p, xi = 1.4, 1.7, 0.9, 7.0
    U = uniform(n, rho, (0.0,) * len(n), p, gamma)
    dt = ro.cfl_dt(U, problem(n, dx, xi=xi, gamma=gamma, cfl_rule=1))
    a = math.sqrt(gamma * p / rho)
    assert (a / xi) * dt / min(dx) == pytest.approx(0.4, rel=1e-13)
    dt0 = ro.cfl_dt(U, problem(n, dx, xi=xi, gamma=gamma))
    if len(n) == 1:
        assert dt == pytest.approx(dt0, rel=1e-14)
    else:
        assert dt > dt0


def test_cfl_scales_with_speeds_and_lengths():
    torch.manual_seed(0)
    n, dx = (12, 9), (0.05, 0.08)
    rho = 1.0 + 0.3 * torch.rand(tuple(reversed(n)), dtype=DT)
    vx, vy = 0.4 * torch.rand_like(rho) - 0.2, 0.4 * torch.rand_like(rho) - 0.2
    P = 0.5 + torch.rand_like(rho)
    gamma = 1.4
    U = torch.stack([rho, rho * vx, rho * vy, P / (gamma - 1) + 0.5 * rho * (vx ** 2 + vy ** 2)])
    dt = ro.cfl_dt(U, problem(n, dx, xi=3.0))
    k = 2.5
    Uk = torch.stack([U[0], k * U[1], k * U[2], k * k * U[3]])  # every speed (V and a) times k
    assert ro.cfl_dt(Uk, problem(n, dx, xi=3.0)) == pytest.approx(dt / k, rel=1e-13)
    assert ro.cfl_dt(U, problem(n, tuple(k * h for h in dx), xi=3.0)) == pytest.approx(k * dt, rel=1e-13)


def _entropy_wave_error(n, variant, xi):
    gamma = 1.4
    x = (torch.arange(n, dtype=DT) + 0.5) / n
    rho = 1.0 + 0.2 * torch.sin(2.0 * math.pi * x)
    U0 = torch.stack([rho, rho, 1.0 / (gamma - 1) + 0.5 * rho])  # u = 1, P = 1: period 1
    prob = problem((n,), (1.0 / n,), xi=xi, variant=variant, gamma=gamma)
    steps = math.ceil(1.0 / ro.cfl_dt(U0, prob))
    U = ro.run(U0, prob, steps, dt=1.0 / steps)
    return float((U[0] - U0[0]).abs().mean())


@pytest.mark.parametrize("variant,xi", [(ro.EULER, 1.0), (ro.PVS, 5.0), (ro.PMS, 5.0)])
def test_entropy_wave_converges_at_second_order(variant, xi):
    err = [_entropy_wave_error(n, variant, xi) for n in (64, 128, 256)]
    orders = [math.log2(err[i] / err[i + 1]) for i in range(2)]
    assert orders[0] > 1.8 and orders[1] > 1.9, (err, orders)


def _entropy_wave_2d_error(axis, variant=ro.EULER, xi=1.0, n=64, m=8):
    """Entropy wave along `axis` on a grid whose cells are 16 times longer
    along the other axis (n cells on [0, 1], m cells on [0, 2])."""
    gamma = 1.4
    nx, ny = (n, m) if axis == 0 else (m, n)
    Lx, Ly = (1.0, 2.0) if axis == 0 else (2.0, 1.0)
    t = (torch.arange(n, dtype=DT) + 0.5) / n
    prof = 1.0 + 0.2 * torch.sin(2.0 * math.pi * t)
    rho = (prof[None, :].expand(ny, nx) if axis == 0 else prof[:, None].expand(ny, nx)).contiguous()
    vx, vy = (1.0, 0.0) if axis == 0 else (0.0, 1.0)
    U0 = torch.stack([rho, rho * vx, rho * vy, 1.0 / (gamma - 1) + 0.5 * rho * (vx * vx + vy * vy)])
    prob = ro.Problem(ndim=2, n=(nx, ny), dx=(Lx / nx, Ly / ny), gamma=gamma, xi=xi, variant=variant,
                      bc=(ro.PERIODIC, ro.PERIODIC), cfl=0.4, vertical=-1, bg_rho=None, bg_p=None, cmax=None)
    steps = math.ceil(1.0 / ro.cfl_dt(U0, prob))
    U = ro.run(U0, prob, steps, dt=1.0 / steps)
    return float((U[0] - U0[0]).abs().mean())


@pytest.mark.parametrize("variant,xi", [(ro.EULER, 1.0), (ro.PVS, 5.0)])
def test_entropy_wave_on_an_anisotropic_grid(variant, xi):
    """Each axis's flux difference is divided by that axis's cell width: the
    wave comes back after one period along x and along y alike (a width
    taken from the other axis moves it 16 times too fast or too slow)."""
    ex = _entropy_wave_2d_error(0, variant, xi)
    ey = _entropy_wave_2d_error(1, variant, xi)
    assert ex < 2e-3, ex
    assert ey == pytest.approx(ex, rel=1e-9)
