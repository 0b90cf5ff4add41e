"""Rayleigh-Taylor workload (the paper's RT test, initial data as printed:
rho1 = 1, rho2 = 10, L = 0.025, eps = 0.01 sin(4 pi x), P = Pc - m_c g_y with
Pc = 1000, g_y = -1, free-slip y walls, periodic x).  The paper prints no
values for it (only max|V_y|(t) plots), so parity with the paper is not
claimed: the CUDA path is checked against the oracle, the unperturbed
hydrostatic state stays at rest, and the reduced forms are compared with the
unreduced (xi = 1) run of the same scheme."""
import math

import pytest
import torch

from oracle import rsst_oracle as ro
from oracle.workload import problem_from
from paper_1812_04135_gb300 import inputs, rsst
from tests.parity import check_precision

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import os
    if not os.path.exists(rsst.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    rsst.lib()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32_pert", 1e-5)])
def test_rt_matches_oracle(precision, tol):
    w = inputs.rayleigh_taylor_2d(64, xi=10.0, variant="pvs")
    s = rsst.Solver(w, precision)
    s.set_state(torch.from_numpy(w["U"]).cuda())
    s.step(5)
    got = s.get_state("cpu")
    s.close()
    prob, U = problem_from(w)
    ref = ro.run(U, prob, 5)
    check_precision(got, ref, w, U, prob, 5, precision, tol)


@pytest.mark.parametrize("precision", ["fp64", "fp32_pert"])
def test_rt_unperturbed_state_stays_at_rest(precision):
    w = inputs.rayleigh_taylor_2d(128, xi=10.0, variant="pvs", amp=0.0)
    s = rsst.Solver(w, precision)
    s.set_state(torch.from_numpy(w["U"]).cuda())
    s.step(500)
    U = s.get_state("cpu")
    t = s.time()
    s.close()
    vmax = float((U[1:3] / U[0]).abs().max())
    assert t > 0.0
    assert vmax < 1e-2, vmax   # the instability itself reaches O(1)


def _vy_history(var, xi, times, n=128, precision="fp32_pert"):
    w = inputs.rayleigh_taylor_2d(n, xi=xi, variant=var)
    s = rsst.Solver(w, precision)
    s.set_state(torch.from_numpy(w["U"]).cuda())
    out = []
    for T in times:
        while s.time() < T:
            s.step(25)
        U = s.get_state("cpu")
        out.append(float((U[2] / U[0]).abs().max()))
    s.close()
    return out


def test_rt_growth_reduced_forms_track_the_unreduced_run():
    """Pressure-reduced forms at xi = 10 follow the unreduced run's
    max|V_y|(t) (within 15 % to t = 1.6; xi = 3 within 8 %); the density-
    reduced DVS form cannot run this ratio-10 interface (Sec. 2.2): it turns
    non-physical early."""
    times = (0.4, 0.8, 1.2, 1.6)
    ref = _vy_history("euler", 1.0, times)
    runs = {(var, xi): _vy_history(var, xi, times) for var, xi in (("pvs", 10.0), ("pms", 10.0), ("pvs", 3.0))}
    print("\nmax|V_y|(t) at t =", times)
    print("  euler xi=1 :", " ".join("%.4f" % v for v in ref))
    for (var, xi), h in runs.items():
        print(f"  {var:5s} xi={xi:g}:", " ".join("%.4f" % v for v in h))
    assert ref[-1] > 20 * ref[0]                 # the instability grows
    for (var, xi), h in runs.items():
        tol = 0.15 if xi > 5 else 0.08
        for r, v in zip(ref, h):
            assert abs(v - r) < tol * r, (var, xi, r, v)
    with pytest.raises(rsst.RsstError) as e:
        _vy_history("dvs", 10.0, (0.4,))
    assert e.value.code == rsst.RSST_ENONPHYSICAL


def _vy_history_at(var, xi, times, n, precision="fp32_pert"):
    """max|V_y| at exactly the given times (adaptive steps, the last one of
    each interval shortened to land on the time)."""
    w = inputs.rayleigh_taylor_2d(n, xi=xi, variant=var)
    s = rsst.Solver(w, precision)
    s.set_state(torch.from_numpy(w["U"]).cuda())
    out = []
    for T in times:
        while True:
            rem = T - s.time()
            if rem <= 1e-12 * T:
                break
            dt = s.dt()
            if dt >= rem:
                s.step(1, rem)
                break
            s.step(max(1, min(int(rem / dt) - 1, 256)))
        U = s.get_state("cuda")
        out.append(float((U[2] / U[0]).abs().max()))
    s.close()
    return out


@pytest.mark.slow
def test_rt_growth_at_1024():
    """The same comparison at 1024^2 (float32 perturbation; the xi = 1 run
    takes ~3e5 steps to t = 1.6, xi = 10 ~3e4): the pressure-reduced forms
    track the unreduced run within the same bounds as at 128^2."""
    times = (0.4, 0.8, 1.2, 1.6)
    ref = _vy_history_at("euler", 1.0, times, 1024)
    runs = {(var, xi): _vy_history_at(var, xi, times, 1024) for var, xi in (("pvs", 10.0), ("pms", 10.0), ("pvs", 3.0))}
    print("\n1024^2 max|V_y|(t) at t =", times)
    print("  euler xi=1 :", " ".join("%.4f" % v for v in ref))
    for (var, xi), h in runs.items():
        print(f"  {var:5s} xi={xi:g}:", " ".join("%.4f" % v for v in h))
    assert ref[-1] > 20 * ref[0]
    for (var, xi), h in runs.items():
        tol = 0.15 if xi > 5 else 0.08
        for r, v in zip(ref, h):
            assert abs(v - r) < tol * r, (var, xi, r, v)
