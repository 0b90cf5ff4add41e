"""The background (hydrostatic profile, wall ghosts, float32 perturbation
tables) along an axis other than the last: the stratified workloads are
transposed so that gravity and the profile lie along x (1D, 2D, 3D) or y
(3D).  These runs take the generic float32 kernel and the background-wall
code of every precision; each is compared with the oracle on the same
transposed data.  The transposition only relabels axes (momentum components
follow their axes), so the physics is the same as the untransposed case."""
import pytest
import torch

from oracle import rsst_oracle as ro
from oracle.workload import problem_from
from paper_1812_04135_gb300 import inputs, rsst
from tests.parity import check_precision, column_1d, permute

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-10, "fp64_df": 1e-10, "fp32_pert": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import os
    if not os.path.exists(rsst.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    rsst.lib()


CASES = {
    "1d_vertical_x": lambda: column_1d(inputs.polytrope_2d(4, 40, xi=20.0, contrast=20.0, amp=1e-2)),
    "2d_vertical_x": lambda: permute(inputs.polytrope_2d(24, 40, xi=20.0, contrast=20.0, amp=1e-2), [1, 0]),
    "3d_vertical_x": lambda: permute(inputs.polytrope_3d(12, 10, 36, xi=50.0, contrast=20.0, amp=1e-2), [2, 0, 1]),
    "3d_vertical_y": lambda: permute(inputs.polytrope_3d(12, 10, 36, xi=50.0, contrast=20.0, amp=1e-2), [0, 2, 1]),
}


@pytest.mark.parametrize("precision", ["fp64", "fp64_df", "fp32_pert"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_background_along_another_axis(name, precision):
    w = CASES[name]()
    prob, U = problem_from(w)
    ref = ro.run(U, prob, 5)
    s = rsst.Solver(w, precision)
    s.set_state(torch.from_numpy(w["U"]).cuda())
    s.step(5)
    got = s.get_state("cpu")
    s.close()
    check_precision(got, ref, w, U, prob, 5, precision, TOL[precision], what=name)
