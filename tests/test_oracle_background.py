"""Reflecting walls with a hydrostatic background (App. B gravity, Sec. 4.6
closed free-slip walls): mirror symmetry is kept, the background-consistent
ghost cells make the hydrostatic residual converge with resolution, and a
gas at rest in a box without gravity stays at rest."""
import numpy as np
import pytest
import torch

from oracle import rsst_oracle as ro
from oracle.workload import problem_from
from paper_1812_04135_gb300 import inputs


def _residual(n):
    w = inputs.polytrope_2d(8, n, xi=20.0, amp=0.0, contrast=20.0)
    prob, U = problem_from(w)
    L = ro.rhs(U, prob)
    # momentum tendency in the vertical direction, scaled by rho g
    return float((L[2] / U[0]).abs().max())


def test_hydrostatic_residual_converges():
    r = [_residual(n) for n in (32, 64, 128)]
    assert r[1] < r[0] and r[2] < r[1]
    assert np.log2(r[1] / r[2]) > 0.9


def test_pure_mirror_wall_would_not_converge():
    """Without the background the wall ghost is a pure mirror, which cannot
    carry the hydrostatic pressure jump: the wall residual stays O(g)."""
    res = []
    for n in (32, 64, 128):
        w = inputs.polytrope_2d(8, n, xi=20.0, amp=0.0, contrast=20.0)
        w["bg_rho"] = None
        w["bg_p"] = None
        prob, U = problem_from(w)
        L = ro.rhs(U, prob)
        res.append(float((L[2] / U[0]).abs().max()))
    assert min(res) > 0.2


def test_mirror_symmetry_about_wall_midplane():
    """A state symmetric under y -> 1 - y (with m_y odd) stays symmetric."""
    n = 16
    w = inputs.random_smooth_state(2, (12, n), xi=4.0, bc=("periodic", "reflect"))
    U = torch.tensor(w["U"])
    U = 0.5 * (U + torch.flip(U, dims=[1]) * torch.tensor([1, 1, -1, 1.0]).reshape(4, 1, 1))
    w["U"] = U.numpy()
    for var in ("pvs", "dms"):
        prob, U0 = problem_from(w, variant=var)
        U1 = ro.run(U0, prob, 5)
        mirrored = torch.flip(U1, dims=[1]) * torch.tensor([1, 1, -1, 1.0]).reshape(4, 1, 1)
        assert torch.allclose(U1, mirrored, rtol=1e-12, atol=1e-13)


def test_rest_state_in_box_stays_at_rest():
    w = inputs.uniform_state(3, (6, 5, 4), vel=(0.0, 0.0, 0.0))
    w["bc"] = ("reflect", "periodic", "reflect")
    for var in ("pvs", "pms"):
        prob, U = problem_from(w, variant=var)
        assert torch.equal(ro.run(U, prob, 3), U)


@pytest.mark.parametrize("order", [[1, 0]])
def test_axis_relabelling_commutes_with_the_step_2d(order):
    """Stepping a stratified box with its axes relabelled (gravity, walls and
    background along x instead of y) equals relabelling the stepped box: the
    oracle treats every axis alike (catches an axis-index slip)."""
    from tests.parity import permute
    w = inputs.polytrope_2d(12, 20, xi=20.0, contrast=20.0, amp=1e-2)
    wt = permute(w, order)
    prob, U = problem_from(w)
    probt, Ut = problem_from(wt)
    a = ro.run(U, prob, 3).numpy()
    b = ro.run(Ut, probt, 3).numpy()
    back = permute(dict(w, U=a), order)["U"]
    assert np.allclose(b, back, rtol=0, atol=1e-12 * np.abs(back).max())


@pytest.mark.parametrize("order", [[2, 0, 1], [0, 2, 1]])
def test_axis_relabelling_commutes_with_the_step_3d(order):
    from tests.parity import permute
    w = inputs.polytrope_3d(8, 6, 20, xi=50.0, contrast=20.0, amp=1e-2)
    wt = permute(w, order)
    prob, U = problem_from(w)
    probt, Ut = problem_from(wt)
    a = ro.run(U, prob, 2).numpy()
    b = ro.run(Ut, probt, 2).numpy()
    back = permute(dict(w, U=a), order)["U"]
    assert np.allclose(b, back, rtol=0, atol=1e-12 * np.abs(back).max())
