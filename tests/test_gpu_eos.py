"""The covolume (Noble-Abel) gas on the float64 device path against the
oracle's general-EOS step (Sec. 3.2: the reduced equations and the pressure
tendency, Eqs. pvs_cons_dpr / pvs_cons_therm, hold for any EOS; the gas is
oracle/eos.py's, selected by rsst_config.covolume).  Tolerance: 1e-10 of each
field's own size, or the oracle's round-off floor (tests/parity.py).  b = 0
is the ideal gas bit for bit; the other precisions and the adjoint refuse a
covolume gas."""
import numpy as np
import pytest
import torch

from oracle import rsst_oracle as ro
from oracle.eos import NobleAbel
from oracle.workload import problem_from
from paper_1812_04135_gb300 import inputs, rsst
from tests.parity import assert_parity

pytestmark = pytest.mark.gpu
SIZES = {1: (300,), 2: (70, 37), 3: (35, 18, 11)}
B = 0.15


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import os
    if not os.path.exists(rsst.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    rsst.lib()


def gpu_run(w, nsteps):
    s = rsst.Solver(w, "fp64")
    try:
        s.set_state(torch.from_numpy(w["U"]).cuda())
        s.step(nsteps)
        return s.get_state("cpu")
    finally:
        s.close()


def check(w, nsteps, what=""):
    prob, U = problem_from(w)
    assert isinstance(prob.gamma, NobleAbel)
    ref = ro.run(U, prob, nsteps)
    assert_parity(gpu_run(w, nsteps), ref, w, U, prob, nsteps, what=what)


@pytest.mark.parametrize("ndim", [1, 2, 3])
@pytest.mark.parametrize("var", ["euler", "dvs", "pvs", "dms", "pms", "pd"])
def test_covolume_gas_all_forms(ndim, var):
    w = inputs.random_smooth_state(ndim, SIZES[ndim], xi=6.0, variant=var)
    w["covolume"] = B
    check(w, 4, what=(ndim, var))


@pytest.mark.parametrize("ndim", [2, 3])
def test_covolume_gas_walls_gravity_background_and_cmax(ndim):
    """Reflecting walls with a hydrostatic-profile background (its energy
    E0 = e(rho0, P0) of the covolume gas), gravity, and the C_max law."""
    w = (inputs.polytrope_2d(40, 70, xi=20.0, contrast=20.0, amp=1e-2) if ndim == 2
         else inputs.polytrope_3d(20, 12, 40, xi=50.0, amp=1e-2, contrast=20.0))
    assert float(np.max(w["bg_rho"])) * 0.02 < 0.5  # rho reaches ~21 at the bottom
    w["covolume"] = 0.02
    check(w, 5, what=ndim)
    w["cmax"] = 0.05
    check(w, 5, what=(ndim, "cmax"))


def test_covolume_changes_the_step_and_zero_is_the_ideal_gas():
    w = inputs.random_smooth_state(2, (40, 30), xi=4.0, variant="pvs")
    ideal = gpu_run(w, 3)
    w0 = dict(w)
    w0["covolume"] = 0.0
    assert torch.equal(gpu_run(w0, 3), ideal)
    w1 = dict(w)
    w1["covolume"] = B
    assert float((gpu_run(w1, 3) - ideal).abs().max()) > 1e-6


def test_adjoint_refuses_a_covolume_gas():
    w = inputs.random_smooth_state(2, (16, 12), xi=3.0)
    w["covolume"] = B
    s = rsst.Solver(w, "fp64")
    try:
        s.set_state(torch.from_numpy(w["U"]).cuda())
        with pytest.raises(rsst.RsstError) as e:
            rsst.rsst_adjoint_record(s.h, 1e-4, 2, 1)
        assert e.value.code == rsst.RSST_EUNSUPPORTED
    finally:
        s.close()


def test_state_beyond_the_covolume_is_flagged():
    """b rho >= 1 is outside the gas: the step flags it as non-physical."""
    w = inputs.random_smooth_state(1, (64,), xi=3.0, variant="pvs")
    w["covolume"] = 1.0 / float(np.min(w["U"][0])) * 1.05
    s = rsst.Solver(w, "fp64")
    try:
        s.set_state(torch.from_numpy(w["U"]).cuda())
        with pytest.raises(rsst.RsstError) as e:
            s.sync()
        assert e.value.code == rsst.RSST_ENONPHYSICAL
    finally:
        s.close()
