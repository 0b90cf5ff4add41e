"""The other reading of the multi-dimensional CFL step (cfl_rule = 1:
dt = C min_d dx_d / max_cells c_tot) through the C ABI, in every precision
and in the batched kernel: the adaptive step and the state after five steps
against the oracle under the same rule, on grids whose cell widths differ
between axes."""
import pytest
import torch

from oracle import rsst_oracle as ro
from oracle.workload import problem_from
from paper_1812_04135_gb300 import inputs, rsst
from tests.parity import check_precision, rel_linf

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-10, "fp64_df": 1e-10, "fp32_pert": 1e-5}
DT_TOL = {"fp64": 1e-12, "fp64_df": 1e-12, "fp32_pert": 1e-6}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import os
    if not os.path.exists(rsst.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    rsst.lib()


CASES = {
    "2d_walls_gravity": lambda: inputs.random_smooth_state(2, (40, 24), xi=5.0, variant="pms",
                                                           bc=("periodic", "reflect"), grav=(0.0, -0.3, 0.0)),
    "2d_stratified": lambda: inputs.polytrope_2d(20, 24, xi=20.0, contrast=20.0, amp=1e-2),
    "3d_stratified": lambda: inputs.polytrope_3d(12, 10, 36, xi=50.0, contrast=20.0, amp=1e-2),
    "1d": lambda: inputs.random_smooth_state(1, (70,), xi=3.0, variant="dvs"),
}


@pytest.mark.parametrize("precision", ["fp64", "fp64_df", "fp32_pert"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_min_width_cfl_rule_matches_oracle(name, precision):
    w = CASES[name]()
    w["cfl_rule"] = 1
    prob, U = problem_from(w)
    assert prob.cfl_rule == 1
    dt_ref = ro.cfl_dt(U, prob)
    ref = ro.run(U, prob, 5)
    s = rsst.Solver(w, precision)
    s.set_state(torch.from_numpy(w["U"]).cuda())
    assert s.dt() == pytest.approx(dt_ref, rel=DT_TOL[precision])
    s.step(5)
    got = s.get_state("cpu")
    s.close()
    check_precision(got, ref, w, U, prob, 5, precision, TOL[precision], what=name)


def test_min_width_cfl_rule_in_the_batched_kernel():
    ws = inputs.batched_runs(count=3, seed=4, max_size=40)
    ws[1] = inputs.polytrope_2d(20, 24, xi=20.0, contrast=20.0, amp=1e-2)
    for w in ws:
        w["cfl_rule"] = 1
    b = rsst.BatchSolver(ws)
    for i, w in enumerate(ws):
        b.set_state(i, torch.from_numpy(w["U"]).cuda())
    b.step(3)
    b.sync()
    for i, w in enumerate(ws):
        prob, U = problem_from(w)
        err = rel_linf(b.get_state(i, "cpu"), ro.run(U, prob, 3), w["gamma"])
        assert max(err) < 1e-5, (i, err)
    b.close()
