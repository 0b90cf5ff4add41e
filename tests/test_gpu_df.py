"""Double-float precision (float32 pairs, 48-bit significand, float32 pipe)
against the float64 oracle at the float64 tolerance, 1e-10 per field."""
import pytest
import torch

from oracle import rsst_oracle as ro
from oracle.workload import problem_from
from paper_1812_04135_gb300 import inputs, rsst
from tests.parity import assert_parity

pytestmark = pytest.mark.gpu
TOL = 1e-10
SIZES = {1: (300,), 2: (70, 37), 3: (35, 18, 11)}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import os
    if not os.path.exists(rsst.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    rsst.lib()


def run(w, nsteps, dt=0.0):
    s = rsst.Solver(w, "fp64_df")
    try:
        s.set_state(torch.from_numpy(w["U"]).cuda())
        s.step(nsteps, dt)
        return s.get_state("cpu")
    finally:
        s.close()


def ref(w, nsteps, dt=None):
    prob, U = problem_from(w)
    return ro.run(U, prob, nsteps, dt=dt)


def check(w, nsteps, tol=TOL, what=""):
    """Own-scale parity at 1e-10, or within the oracle's round-off floor for
    the double-float unit round-off 2^-48 (tests/parity.py)."""
    prob, U = problem_from(w)
    assert_parity(run(w, nsteps), ro.run(U, prob, nsteps), w, U, prob, nsteps, precision="fp64_df", tol=tol,
                  what=what)


@pytest.mark.parametrize("ndim", [1, 2, 3])
@pytest.mark.parametrize("var", ["euler", "dvs", "pvs", "dms", "pms", "pd"])
def test_periodic_all_forms(ndim, var):
    check(inputs.random_smooth_state(ndim, SIZES[ndim], xi=6.0, variant=var), 4, what=(ndim, var))


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_walls_gravity_and_cmax(ndim):
    bc = ("reflect", "periodic", "reflect")[:ndim] if ndim > 1 else ("reflect",)
    grav = (0.3, -0.8, 0.5)[:ndim] + (0.0,) * (3 - ndim)
    w = inputs.random_smooth_state(ndim, SIZES[ndim], xi=5.0, variant="pms", bc=bc, grav=grav)
    check(w, 4, what=ndim)
    w["cmax"] = 0.35
    check(w, 4, what=(ndim, "cmax"))


def test_stratified_background():
    check(inputs.polytrope_2d(40, 70, xi=20.0, contrast=20.0, amp=1e-2), 6)
    check(inputs.polytrope_3d(20, 12, 40, xi=50.0, amp=1e-2, contrast=20.0), 5)


def test_shear_layer_full_size_and_many_steps():
    w = inputs.shear_layer_2d()
    check(w, 3)
    w = inputs.sound_wave_1d(256, xi=10.0, variant="pvs")
    check(w, 200)


def test_momentum_conserved_and_flag():
    w = inputs.shear_layer_2d(256, 256, xi=30.0, variant="pms")
    s = rsst.Solver(w, "fp64_df")
    s.set_state(torch.from_numpy(w["U"]).cuda())
    s0 = s.sums()
    s.step(200)
    s1 = s.sums()
    U = torch.from_numpy(w["U"])
    scale_m = float(U[1].abs().sum() + U[2].abs().sum()) / (256 * 256)
    for k in (1, 2):
        assert abs(s1[k] - s0[k]) < 1e-12 * scale_m * 200, (k, s0[k], s1[k])
    s.close()
    w = inputs.contact_1d(256, xi=10.0, variant="dvs")
    s = rsst.Solver(w, "fp64_df")
    s.set_state(torch.from_numpy(w["U"]).cuda())
    s.step(3)
    with pytest.raises(rsst.RsstError) as e:
        s.sync()
    assert e.value.code == rsst.RSST_ENONPHYSICAL
    s.close()


@pytest.mark.parametrize("n", [19456, 20011])
def test_long_1d_lines_use_wide_tiles(n):
    check(inputs.random_smooth_state(1, (n,), xi=6.0, variant="dms"), 3, what=n)
