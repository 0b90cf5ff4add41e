"""Failure detection on the device without a GPU fault.

Every wait of the TMA-staged kernels is bounded.  The library's test hook
makes each tile of a TMA-staged kernel (2D float32 perturbation: after its
own copy has landed; 3D float32 z-march and 2D/3D float64: with a copy still
in flight) also wait on a shared-memory barrier that nothing completes, with
a 1 ms limit.  The wait runs out, the kernel sets the run's timeout flag,
waits (bounded) for any copy it issued, and returns; the next synchronous
call must return RSST_ETIMEOUT (not RSST_ENONPHYSICAL), the context must stay
usable, and a fresh state must then step to the oracle's result."""
import pytest
import torch

from oracle import rsst_oracle as ro
from oracle.workload import problem_from
from paper_1812_04135_gb300 import inputs, rsst
from tests.parity import rel_linf

pytestmark = pytest.mark.gpu
LIMIT_NS = 1_000_000  # 1 ms


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import os
    if not os.path.exists(rsst.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    rsst.lib()


def _oracle(w, nsteps):
    prob, U = problem_from(w)
    return ro.run(U, prob, nsteps)


@pytest.mark.parametrize("stage_steps", [1, 2])
def test_single_run_wait_runs_out_and_is_reported(stage_steps):
    w = inputs.shear_layer_2d(200, 44, xi=30.0, variant="pvs")
    U = torch.from_numpy(w["U"]).cuda()
    s = rsst.Solver(w, "fp32_pert")
    try:
        s.set_state(U)
        rsst.rsst_debug_stall_wait(s.h, LIMIT_NS)
        s.step(stage_steps)
        with pytest.raises(rsst.RsstError) as e:
            s.sync()
        assert e.value.code == rsst.RSST_ETIMEOUT, str(e.value)
        assert "gave up" in str(e.value)
        # the flag is sticky until a new state is loaded
        with pytest.raises(rsst.RsstError) as e2:
            s.dt()
        assert e2.value.code == rsst.RSST_ETIMEOUT
        # the context still works: a fresh state steps to the oracle's result
        rsst.rsst_debug_stall_wait(s.h, 0)
        s.set_state(U)
        s.step(3)
        err = rel_linf(s.get_state("cpu"), _oracle(w, 3), w["gamma"])
        assert max(err) < 1e-5, err
    finally:
        s.close()
    torch.cuda.synchronize()


def test_3d_wait_runs_out_drains_and_is_reported():
    """The 3D z-march: the test wait runs out after the first planes have
    landed, with the next plane's copy issued; the kernel drains it, flags
    the run and returns.  A fresh state then steps to the oracle's result."""
    w = inputs.polytrope_3d(40, 12, 37, xi=50.0, amp=1e-3, contrast=20.0)
    U = torch.from_numpy(w["U"]).cuda()
    s = rsst.Solver(w, "fp32_pert")
    try:
        s.set_state(U)
        rsst.rsst_debug_stall_wait(s.h, LIMIT_NS)
        s.step(1)
        with pytest.raises(rsst.RsstError) as e:
            s.sync()
        assert e.value.code == rsst.RSST_ETIMEOUT, str(e.value)
        rsst.rsst_debug_stall_wait(s.h, 0)
        s.set_state(U)
        s.step(2)
        err = rel_linf(s.get_state("cpu"), _oracle(w, 2), w["gamma"])
        assert max(err) < 1e-5, err
    finally:
        s.close()


@pytest.mark.parametrize("case", ["shear2d", "polytrope3d"])
def test_fp64_wait_runs_out_drains_and_is_reported(case):
    """The float64 stage kernel (2D and 3D halo tiles by TMA): the test wait
    runs out with the tile's copy in flight; the kernel waits for it, flags
    the run and returns.  A fresh state then steps to the oracle's result."""
    if case == "shear2d":
        w = inputs.shear_layer_2d(72, 40, xi=30.0, variant="pvs")
    else:
        w = inputs.polytrope_3d(24, 16, 20, xi=50.0, amp=1e-3, contrast=20.0)
    U = torch.from_numpy(w["U"]).cuda()
    s = rsst.Solver(w, "fp64")
    try:
        s.set_state(U)
        rsst.rsst_debug_stall_wait(s.h, LIMIT_NS)
        s.step(1)
        with pytest.raises(rsst.RsstError) as e:
            s.sync()
        assert e.value.code == rsst.RSST_ETIMEOUT, str(e.value)
        rsst.rsst_debug_stall_wait(s.h, 0)
        s.set_state(U)
        s.step(2)
        err = rel_linf(s.get_state("cpu"), _oracle(w, 2), w["gamma"])
        assert max(err) < 1e-10, err
    finally:
        s.close()


def test_stall_hook_validation():
    w = inputs.shear_layer_2d(64, 32, xi=30.0, variant="pvs")
    s = rsst.Solver(w, "fp32_pert")
    try:
        for bad in (-1, 2_000_000_000):
            with pytest.raises(rsst.RsstError) as e:
                rsst.rsst_debug_stall_wait(s.h, bad)
            assert e.value.code == rsst.RSST_EINVAL
    finally:
        s.close()
    # kernels without a TMA-staged tile have no test wait: double-float, 1D
    for ws, precision in ((w, "fp64_df"), (inputs.sound_wave_1d(256, xi=10.0), "fp64")):
        s = rsst.Solver(ws, precision)
        try:
            with pytest.raises(rsst.RsstError) as e:
                rsst.rsst_debug_stall_wait(s.h, LIMIT_NS)
            assert e.value.code == rsst.RSST_EUNSUPPORTED
        finally:
            s.close()


def test_batched_wait_runs_out_and_names_a_run():
    ws = inputs.batched_runs(count=5, seed=4, sizes=(40, 64, 72, 96, 130, 33))
    b = rsst.BatchSolver(ws)
    try:
        states = [torch.from_numpy(w["U"]).cuda() for w in ws]
        for i, U in enumerate(states):
            b.set_state(i, U)
        rsst.rsst_batch_debug_stall_wait(b.b, 2, LIMIT_NS)
        b.step(1)
        with pytest.raises(rsst.RsstError) as e:
            b.sync()
        assert e.value.code == rsst.RSST_ETIMEOUT, str(e.value)
        assert "run" in str(e.value)
        rsst.rsst_batch_debug_stall_wait(b.b, 2, 0)
        for i, U in enumerate(states):
            b.set_state(i, U)
        b.step(3)
        b.sync()
        for i, w in enumerate(ws):
            err = rel_linf(b.get_state(i, "cpu"), _oracle(w, 3), w["gamma"])
            assert max(err) < 1e-5, (i, err)
    finally:
        b.close()
