"""Edge cases of the CUDA path through the C ABI: the smallest grids the
library accepts (two cells along an axis, where every ghost cell wraps or
mirrors an interior cell), the degenerate xi = 1 where every reduced form is
the Euler step (f = 1 - 1/xi^2 = 0 exactly, Sec. 3.2), a uniform state that
stays exactly steady, and the full batched workload on sampled runs."""
import numpy as np
import pytest
import torch

from oracle import rsst_oracle as ro
from oracle.workload import problem_from
from paper_1812_04135_gb300 import inputs, rsst
from tests.parity import check_precision, rel_linf

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-10, "fp64_df": 1e-10, "fp32_pert": 1e-5}
FORMS = ["euler", "dvs", "pvs", "dms", "pms", "pd"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import os
    if not os.path.exists(rsst.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    rsst.lib()


def gpu_run(w, precision, nsteps, dt=0.0):
    s = rsst.Solver(w, precision)
    try:
        s.set_state(torch.from_numpy(w["U"]).cuda())
        s.step(nsteps, dt)
        return s.get_state("cpu")
    finally:
        s.close()


@pytest.mark.parametrize("precision", ["fp64", "fp64_df", "fp32_pert"])
@pytest.mark.parametrize("n,bc", [((2,), ("periodic",)), ((2,), ("reflect",)), ((2, 2), ("periodic", "reflect")),
                                  ((5, 2), ("reflect", "periodic")), ((2, 3, 2), ("periodic", "reflect", "periodic")),
                                  ((3, 2, 4), ("reflect", "reflect", "reflect"))])
def test_smallest_grids(precision, n, bc):
    """n = 2 along an axis: both ghost layers come from the two interior cells."""
    w = inputs.random_smooth_state(len(n), n, xi=4.0, variant="pvs", bc=bc)
    prob, U = problem_from(w)
    ref = ro.run(U, prob, 3)
    check_precision(gpu_run(w, precision, 3), ref, w, U, prob, 3, precision, TOL[precision], what=(n, bc))


@pytest.mark.parametrize("precision", ["fp64", "fp64_df", "fp32_pert"])
def test_xi_one_reduces_every_form_to_euler_bitwise(precision):
    """At xi = 1 the factor f = 1 - 1/xi^2 is exactly 0, so every reduced form
    produces the Euler state bit for bit, with walls and gravity."""
    base = inputs.random_smooth_state(2, (37, 21), xi=1.0, variant="euler", bc=("periodic", "reflect"),
                                      grav=(0.0, -0.4, 0.0))
    ref = gpu_run(base, precision, 4)
    for var in FORMS[1:]:
        w = dict(base)
        w["variant"] = var
        assert torch.equal(gpu_run(w, precision, 4), ref), (precision, var)


@pytest.mark.parametrize("precision", ["fp64", "fp64_df", "fp32_pert"])
@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_uniform_moving_state_is_exactly_steady(precision, ndim):
    """A uniform state (with velocity) has zero tendency in every form: after
    10 adaptive steps the stored state is unchanged bit for bit (compared
    with the state read back before stepping, which is the input rounded to
    the storage precision)."""
    n = {1: (40,), 2: (24, 18), 3: (12, 10, 9)}[ndim]
    for var in FORMS:
        w = inputs.uniform_state(ndim, n, xi=10.0, variant=var)
        s = rsst.Solver(w, precision)
        s.set_state(torch.from_numpy(w["U"]).cuda())
        before = s.get_state("cpu")
        s.step(10)
        after = s.get_state("cpu")
        s.close()
        assert torch.equal(after, before), (precision, ndim, var)


def test_full_batched_workload_sampled_runs():
    """All 64 runs of the batched workload (25 M cells) take one persistent
    step; the largest, the smallest and four seeded runs are compared with the
    oracle element by element."""
    ws = inputs.batched_runs(count=64, seed=4)
    b = rsst.BatchSolver(ws)
    for i, w in enumerate(ws):
        b.set_state(i, torch.from_numpy(w["U"]).cuda())
    b.step(1)
    b.sync()
    cells = [int(np.prod(w["n"])) for w in ws]
    picks = {int(np.argmax(cells)), int(np.argmin(cells))}
    picks |= {int(d % np.uint64(64)) for d in inputs.splitmix64(91, 4)}
    for i in sorted(picks):
        w = ws[i]
        prob, U = problem_from(w)
        err = rel_linf(b.get_state(i, "cpu"), ro.run(U, prob, 1), w["gamma"])
        assert max(err) < 1e-5, (i, w["n"], w["xi"], err)
    b.close()


@pytest.mark.parametrize("precision", ["fp64", "fp64_df", "fp32_pert"])
def test_zero_steps_and_rejected_calls_change_nothing(precision):
    """step(0), and calls the library rejects (negative nsteps, non-finite dt),
    launch no kernel and leave the state, the time and the next dt as they
    were.  A float64 state comes back bit for bit from set/get."""
    w = inputs.polytrope_2d(20, 24, xi=20.0, contrast=20.0, amp=1e-2)
    s = rsst.Solver(w, precision)
    U0 = torch.from_numpy(w["U"]).cuda()
    s.set_state(U0)
    before, dt0, n0 = s.get_state("cpu"), s.dt(), s.launches()
    if precision == "fp64":
        assert torch.equal(before, U0.cpu())
    s.step(0)
    for bad in [dict(nsteps=-1), dict(nsteps=1, dt=float("nan")), dict(nsteps=1, dt=float("inf"))]:
        with pytest.raises(rsst.RsstError) as e:
            s.step(**bad)
        assert e.value.code == rsst.RSST_EINVAL
    assert s.launches() == n0
    assert torch.equal(s.get_state("cpu"), before)
    assert s.time() == 0.0 and s.dt() == dt0
    s.close()


def test_batch_zero_steps_change_nothing():
    ws = small_batch_runs()
    b = rsst.BatchSolver(ws)
    for i, w in enumerate(ws):
        b.set_state(i, torch.from_numpy(w["U"]).cuda())
    before = [b.get_state(i, "cpu") for i in range(len(ws))]
    n0 = b.launches()
    b.step(0)
    b.step_looped(0)
    with pytest.raises(rsst.RsstError):
        b.step(-1)
    assert b.launches() == n0
    for i in range(len(ws)):
        assert torch.equal(b.get_state(i, "cpu"), before[i])
    b.close()


def small_batch_runs():
    return inputs.batched_runs(count=3, seed=4, max_size=40)
