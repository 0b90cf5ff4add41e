"""Graph-replayed step blocks (rsst_set_graph_steps) give the same state,
CFL step and simulated time as plain launches, bit for bit, in every
precision and dimension, with adaptive and fixed dt and step counts that
are not multiples of the block."""
import numpy as np
import pytest
import torch

from paper_1812_04135_gb300 import inputs, rsst

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import os
    if not os.path.exists(rsst.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    rsst.lib()


def run(w, precision, k, plan):
    s = rsst.Solver(w, precision)
    s.set_graph_steps(k)
    s.set_state(torch.from_numpy(w["U"]).cuda())
    for n, dt in plan:
        s.step(n, dt)
    out = s.get_state("cpu")
    res = (out, s.dt(), s.time(), s.launches())
    s.close()
    return res


CASES = [
    ("sound1d", lambda: inputs.sound_wave_1d(256, xi=10.0, variant="pvs"), ["fp64", "fp64_df"]),
    ("shear2d", lambda: inputs.shear_layer_2d(64, 48, xi=30.0, variant="pvs", ratio=10.0),
     ["fp64", "fp32_pert", "fp64_df"]),
    ("polytrope3d", lambda: inputs.polytrope_3d(16, 12, 40, xi=50.0, contrast=20.0, variant="pms"),
     ["fp64", "fp32_pert", "fp64_df"]),
]


@pytest.mark.parametrize("name,make,precs", CASES)
def test_graph_blocks_equal_plain_launches(name, make, precs):
    w = make()
    for prec in precs:
        plan = [(37, 0.0), (1, 0.0), (20, 0.0)]
        ref = run(w, prec, 0, plan)
        for k in (2, 16):
            got = run(w, prec, k, plan)
            assert torch.equal(got[0], ref[0]), (name, prec, k)
            assert got[1] == ref[1] and got[2] == ref[2], (name, prec, k)
            assert got[3] == ref[3], (name, prec, k)  # launch count covers the replayed kernels


def test_fixed_dt_change_recaptures():
    w = inputs.shear_layer_2d(64, 64, xi=30.0, variant="dvs", ratio=3.0)
    plan = [(16, 1e-4), (16, 2e-4), (32, 1e-4), (5, 0.0), (16, 0.0)]
    ref = run(w, "fp64", 0, plan)
    got = run(w, "fp64", 16, plan)
    assert torch.equal(got[0], ref[0])
    assert got[2] == ref[2]


def test_set_graph_steps_validation():
    w = inputs.sound_wave_1d(64, xi=1.0, variant="euler")
    s = rsst.Solver(w, "fp64")
    with pytest.raises(rsst.RsstError):
        s.set_graph_steps(3)
    with pytest.raises(rsst.RsstError):
        s.set_graph_steps(-2)
    s.set_graph_steps(0)
    s.close()
