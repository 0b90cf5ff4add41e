"""Discrete adjoint of the float64 step (CUDA, through the C ABI) against the
oracle's reverse-mode derivative of its own step, against central finite
differences of the GPU forward run, and through torch.autograd."""
import math

import numpy as np
import pytest
import torch

from oracle import adjoint as adj
from oracle import rsst_oracle as ro
from oracle.workload import problem_from
from paper_1812_04135_gb300 import inputs, rsst

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import os
    if not os.path.exists(rsst.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    rsst.lib()


def gpu_adjoint(w, dt, nsteps, every, lam_final):
    s = rsst.Solver(w, "fp64")
    s.set_state(torch.from_numpy(w["U"]).cuda())
    rsst.rsst_adjoint_record(s.h, dt, nsteps, every)
    lam = lam_final.clone().cuda().contiguous()
    dxi = 0.0
    for seg in reversed(range(rsst.rsst_adjoint_segments(s.h))):
        dxi += rsst.rsst_adjoint_step(s.h, seg, lam)
    UN = s.get_state("cpu")
    s.close()
    return UN, lam.cpu(), dxi


def close(a, b, rtol):
    scale = float(b.abs().max())
    return float((a - b).abs().max()) <= rtol * scale


CASES = [
    ("polytrope2d", lambda: inputs.polytrope_2d(20, 24, xi=20.0, contrast=20.0, amp=1e-2)),
    ("smooth1d_reflect", lambda: inputs.random_smooth_state(1, (40,), xi=4.0, bc=("reflect",), grav=(0.7, 0, 0))),
    ("smooth2d_periodic", lambda: inputs.random_smooth_state(2, (18, 14), xi=6.0)),
    ("smooth3d_mixed", lambda: inputs.random_smooth_state(3, (10, 8, 9), xi=5.0, bc=("periodic", "reflect", "reflect"),
                                                          grav=(0.0, 0.3, -0.6))),
]


@pytest.mark.parametrize("name,make", CASES)
@pytest.mark.parametrize("var", ["euler", "dvs", "pvs", "dms", "pms", "pd"])
def test_one_step_vjp_matches_oracle(name, make, var):
    w = make()
    w["variant"] = var
    prob, U = problem_from(w)
    dt = 0.5 * ro.cfl_dt(U, prob)
    lam = torch.tensor(inputs.uniform_pm1(99, U.numel()).reshape(U.shape))
    gU, gxi = adj.step_vjp(U, lam, dt, prob)
    _, got, dxi = gpu_adjoint(w, dt, 1, 1, lam)
    assert close(got, gU, 1e-10), (name, var, float((got - gU).abs().max()), float(gU.abs().max()))
    assert dxi == pytest.approx(gxi, rel=1e-9, abs=1e-12 * abs(float(gU.abs().max())))


def test_segments_match_oracle_adjoint_run():
    w = inputs.polytrope_2d(24, 32, xi=20.0, contrast=20.0, amp=1e-2)
    prob, U = problem_from(w)
    dt = ro.cfl_dt(U, prob)
    J, UN, lam0, dxi = adj.adjoint_run(U, prob, 7, dt, 3)
    lamN = ro.kinetic_energy_gradient(UN, prob)
    gUN, got, gdxi = gpu_adjoint(w, dt, 7, 3, lamN)
    assert close(gUN, UN, 1e-13)
    assert close(got, lam0, 1e-9)
    assert gdxi == pytest.approx(dxi, rel=1e-8)


def test_kinetic_energy_and_gradient():
    w = inputs.random_smooth_state(2, (30, 20), xi=3.0)
    prob, U = problem_from(w)
    s = rsst.Solver(w, "fp64")
    s.set_state(torch.from_numpy(w["U"]).cuda())
    g = torch.empty_like(U).cuda()
    J = rsst.rsst_kinetic_energy(s.h, g)
    s.close()
    assert J == pytest.approx(float(ro.kinetic_energy(U, prob)), rel=1e-13)
    assert close(g.cpu(), ro.kinetic_energy_gradient(U, prob), 1e-14)


@pytest.mark.parametrize("ndim,n,dx", [(1, (40,), (0.3,)), (2, (30, 20), (0.1, 0.4)), (3, (12, 10, 9), (0.2, 0.5, 0.125))])
def test_kinetic_energy_of_a_uniform_moving_gas(ndim, n, dx):
    """The device functional against its closed form, 1/2 rho |V|^2 times the
    domain volume, for a gas moving uniformly (no oracle involved)."""
    rho, V, E = 2.5, (0.3, -0.7, 1.1)[:ndim], 9.0
    w = inputs.random_smooth_state(ndim, n, xi=3.0)
    shape = tuple(reversed(n))
    w["U"] = np.ascontiguousarray(np.stack([np.full(shape, rho)] + [np.full(shape, rho * V[d]) for d in range(ndim)]
                                           + [np.full(shape, E)]))
    w["dx"] = tuple(dx)
    volume = float(np.prod([n[d] * dx[d] for d in range(ndim)]))
    s = rsst.Solver(w, "fp64")
    s.set_state(torch.from_numpy(w["U"]).cuda())
    J = rsst.rsst_kinetic_energy(s.h)
    s.close()
    assert J == pytest.approx(0.5 * rho * sum(v * v for v in V) * volume, rel=1e-13)


def test_autograd_function():
    w = inputs.polytrope_2d(16, 24, xi=20.0, contrast=20.0, amp=1e-2)
    prob, U = problem_from(w)
    dt = ro.cfl_dt(U, prob)
    s = rsst.Solver(w, "fp64")
    U0 = torch.from_numpy(w["U"]).cuda().requires_grad_(True)
    xi = torch.tensor(w["xi"], dtype=torch.float64, requires_grad=True)
    UN = rsst.rsst_run(U0, xi, s, dt, 5, 2)
    m2 = UN[1] ** 2 + UN[2] ** 2
    J = (0.5 * m2 / UN[0]).sum() * prob.cell_volume()
    J.backward()
    Jo, _, lam0, dxi = adj.adjoint_run(U, prob, 5, dt, 2)
    assert float(J.detach()) == pytest.approx(Jo, rel=1e-12)
    assert close(U0.grad.cpu(), lam0, 1e-9)
    assert float(xi.grad) == pytest.approx(dxi, rel=1e-8)
    s.close()


def test_adjoint_workload_full_size():
    """2D 256^2 stratified box (contrast 20, xi = 20), 400 steps, checkpoint
    every 20: gradient of the final kinetic energy with respect to the
    initial density (32 seeded cells, 4 seeded whole-field directions) and
    xi, against central differences of the GPU forward run and the oracle
    adjoint."""
    w = inputs.polytrope_2d(256, 256, xi=20.0, contrast=20.0, amp=1e-3)
    prob, U = problem_from(w)
    dt = ro.cfl_dt(U, prob)
    nsteps, every = 400, 20
    s = rsst.Solver(w, "fp64")
    s.set_state(torch.from_numpy(w["U"]).cuda())
    rsst.rsst_adjoint_record(s.h, dt, nsteps, every)
    gN = torch.empty(U.shape, dtype=torch.float64, device="cuda")
    J = rsst.rsst_kinetic_energy(s.h, gN)
    lam = gN.clone()
    dxi = 0.0
    for seg in reversed(range(rsst.rsst_adjoint_segments(s.h))):
        dxi += rsst.rsst_adjoint_step(s.h, seg, lam)
    lam = lam.cpu()
    assert J > 0

    def J_of(Uinit, xi=None):
        ww = dict(w)
        if xi is not None:
            ww["xi"] = xi
        t = rsst.Solver(ww, "fp64")
        t.set_state(Uinit.cuda())
        t.step(nsteps, dt)
        val = rsst.rsst_kinetic_energy(t.h)
        t.close()
        return val

    U0 = torch.from_numpy(w["U"])
    draws = inputs.splitmix64(77, 32)
    cells = [(int(d % np.uint64(256 * 256)) // 256, int(d % np.uint64(256 * 256)) % 256) for d in draws]
    # the oracle's own discrete adjoint (exact up to rounding): sampled cells and xi
    Jo, _, lam0, dxio = adj.adjoint_run(U, prob, nsteps, dt, every)
    assert J == pytest.approx(Jo, rel=1e-9)
    scale = float(lam0[0].abs().max())
    worst = max(abs(float(lam[0, j, i]) - float(lam0[0, j, i])) for (j, i) in cells) / scale
    print("adjoint vs oracle adjoint: max err / max|grad| = %.2e; dJ/dxi %.10e vs %.10e" % (worst, dxi, dxio))
    assert worst < 1e-8
    assert dxi == pytest.approx(dxio, rel=1e-7)
    # Central differences (eps = 1e-6 relative).  The scheme is piecewise
    # smooth (MC branches, the LLF max): over 400 steps a +-h perturbation
    # moves some cells across a branch boundary, so the difference quotient
    # averages one-sided derivatives while the adjoint follows the forward
    # branch; most cells agree to ~1e-4, a few to ~1e-2.
    rel = []
    for (j, i) in cells:
        h = 1e-6 * float(U0[0, j, i])
        Up = U0.clone(); Up[0, j, i] += h
        Um = U0.clone(); Um[0, j, i] -= h
        fd = (J_of(Up) - J_of(Um)) / (2 * h)
        g = float(lam[0, j, i])
        rel.append(abs(fd - g) / abs(g))
    rel = np.array(rel)
    print("adjoint vs central differences: median rel err %.2e, max %.2e, within 1e-3: %d/32"
          % (np.median(rel), rel.max(), int((rel < 1e-3).sum())))
    assert np.median(rel) < 1e-3 and (rel < 1e-2).sum() >= 28, rel
    hx = 1e-6 * w["xi"]
    fdx = (J_of(U0, w["xi"] + hx) - J_of(U0, w["xi"] - hx)) / (2 * hx)
    print("dJ/dxi adjoint %.10e  central difference %.10e" % (dxi, fdx))
    assert dxi == pytest.approx(fdx, rel=1e-2)
    # Four seeded directions d in the initial density field (d = U[-1,1) times
    # the local density): central difference of J(rho0 + eps d) against
    # lam . d.  Measured 1.5e-5 .. 2.5e-4 at eps = 1e-8 (3e-3 at 1e-7, where
    # more cells cross a branch boundary).
    for k in range(4):
        d = torch.tensor(inputs.uniform_pm1(500 + k, 256 * 256).reshape(256, 256)) * U0[0]
        eps = 1e-8
        Up = U0.clone(); Up[0] += eps * d
        Um = U0.clone(); Um[0] -= eps * d
        fd = (J_of(Up) - J_of(Um)) / (2 * eps)
        g = float((lam[0] * d).sum())
        print("direction %d: adjoint %.10e central difference %.10e" % (k, g, fd))
        assert fd == pytest.approx(g, rel=2e-3)
    s.close()


@pytest.mark.parametrize("var", ["pvs", "dms"])
def test_one_step_vjp_cmax(var):
    """Adjoint under the C_max law: the state gradient includes d xi / d a;
    xi is not a parameter then, so dJ/dxi is zero."""
    w = inputs.polytrope_2d(20, 24, xi=1.0, contrast=20.0, amp=1e-2)
    w["variant"] = var
    w["cmax"] = 0.05
    prob, U = problem_from(w)
    dt = 0.5 * ro.cfl_dt(U, prob)
    lam = torch.tensor(inputs.uniform_pm1(98, U.numel()).reshape(U.shape))
    gU, _ = adj.step_vjp(U, lam, dt, prob)
    _, got, dxi = gpu_adjoint(w, dt, 1, 1, lam)
    assert close(got, gU, 1e-10)
    assert dxi == 0.0


@pytest.mark.parametrize("name,make", CASES)
def test_density_gradient_at_fixed_velocity_and_pressure(name, make):
    """rsst_adjoint_rho_fixed_vp on the device against the oracle's chain rule:
    on the same gradient (the kernel alone, to rounding), and on the GPU
    adjoint's gradient against the oracle adjoint's (the whole chain)."""
    w = make()
    prob, U = problem_from(w)
    U = ro.run(U, prob, 2)  # some motion, so V . lam_m and |V|^2 lam_E matter
    w = dict(w)
    w["U"] = U.numpy().copy()
    dt = ro.cfl_dt(U, prob)
    J, UN, lam0, dxi = adj.adjoint_run(U, prob, 5, dt, 2)
    want = adj.rho_gradient_fixed_vp(U, lam0, prob.gamma)
    Ud, ld = U.cuda().contiguous(), lam0.cuda().contiguous()
    out = torch.empty(tuple(U.shape[1:]), dtype=torch.float64, device="cuda")
    rsst.rsst_adjoint_rho_fixed_vp(Ud, ld, out)
    torch.cuda.synchronize()
    assert close(out.cpu(), want, 1e-14)
    _, glam, _ = gpu_adjoint(w, dt, 5, 2, ro.kinetic_energy_gradient(UN, prob))
    rsst.rsst_adjoint_rho_fixed_vp(Ud, glam.cuda().contiguous(), out)
    torch.cuda.synchronize()
    assert close(out.cpu(), want, 1e-9)
