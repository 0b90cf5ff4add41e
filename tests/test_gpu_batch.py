"""Batched float32-perturbation runs (one persistent kernel per stage over
the ragged tile list of all runs) against the float64 oracle per run, against
the looped single-run launches, and the autotuner's save/restore."""
import pytest
import torch

from oracle import rsst_oracle as ro
from oracle.workload import problem_from
from paper_1812_04135_gb300 import inputs, rsst
from tests.parity import rel_linf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import os
    if not os.path.exists(rsst.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    rsst.lib()


def small_batch(count=7):
    # uneven sizes with ragged tiles for every candidate tile shape
    return inputs.batched_runs(count=count, seed=4, sizes=(40, 64, 72, 96, 130, 33))


def test_batch_matches_oracle_per_run():
    ws = small_batch()
    b = rsst.BatchSolver(ws)
    for i, w in enumerate(ws):
        b.set_state(i, torch.from_numpy(w["U"]).cuda())
    b.step(5)
    b.sync()
    for i, w in enumerate(ws):
        prob, U = problem_from(w)
        ref = ro.run(U, prob, 5)
        err = rel_linf(b.get_state(i, "cpu"), ref, w["gamma"])
        assert max(err) < 1e-5, (i, w["n"], w["xi"], err)
    b.close()


def test_batch_matches_looped_single_runs_and_dt():
    ws = small_batch()
    a = rsst.BatchSolver(ws)
    c = rsst.BatchSolver(ws)
    for i, w in enumerate(ws):
        a.set_state(i, torch.from_numpy(w["U"]).cuda())
        c.set_state(i, torch.from_numpy(w["U"]).cuda())
    a.step(6)
    c.step_looped(6)
    da, dc = a.dts(), c.dts()
    for i, w in enumerate(ws):
        x, y = a.get_state(i, "cpu"), c.get_state(i, "cpu")
        assert max(rel_linf(x, y, w["gamma"])) < 1e-6, i
        assert da[i] == pytest.approx(dc[i], rel=1e-6)
    assert a.launches() == 12 and c.launches() == 12 * len(ws)
    a.close()
    c.close()


def test_autotune_keeps_the_state_and_picks_a_shape():
    ws = small_batch(5)
    b = rsst.BatchSolver(ws)
    for i, w in enumerate(ws):
        b.set_state(i, torch.from_numpy(w["U"]).cuda())
    before = [b.get_state(i, "cpu") for i in range(len(ws))]
    choice, ms = b.autotune(2)
    assert 0 <= choice < 6 and ms > 0
    assert b.tile_shape() in [(64, 32), (32, 32), (64, 16), (128, 16), (64, 24), (128, 8)]
    for i in range(len(ws)):
        assert torch.equal(b.get_state(i, "cpu"), before[i])
    b.step(3)
    b.sync()
    b.close()


@pytest.mark.parametrize("choice_shape", [0, 1, 2, 3, 4, 5])
def test_every_tile_shape_is_correct(choice_shape, monkeypatch, tmp_path):
    """Force each candidate through the tuning cache and check the result."""
    ws = small_batch(4)
    key_b = rsst.BatchSolver(ws)
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("RSST_TUNE_CACHE", str(cache))
    for i, w in enumerate(ws):
        key_b.set_state(i, torch.from_numpy(w["U"]).cuda())
    key_b.autotune(1)                                 # writes "<signature> <best>"
    sig = cache.read_text().split()[0]
    cache.write_text(f"{sig} {choice_shape}\n")
    key_b.close()
    b = rsst.BatchSolver(ws)
    for i, w in enumerate(ws):
        b.set_state(i, torch.from_numpy(w["U"]).cuda())
    choice, _ = b.autotune(1)
    assert choice == choice_shape
    b.step(3)
    for i, w in enumerate(ws):
        prob, U = problem_from(w)
        ref = ro.run(U, prob, 3)
        assert max(rel_linf(b.get_state(i, "cpu"), ref, w["gamma"])) < 1e-5, (choice_shape, i)
    b.close()


def test_batch_cmax_law_matches_oracle():
    """Runs under the C_max law (Eq. cx: xi from the local sound speed) in
    the persistent batch kernel, each against the oracle."""
    ws = small_batch(5)
    for w in ws:
        w["cmax"] = 0.3
        w["xi"] = 1.0
    b = rsst.BatchSolver(ws)
    for i, w in enumerate(ws):
        b.set_state(i, torch.from_numpy(w["U"]).cuda())
    b.step(4)
    b.sync()
    for i, w in enumerate(ws):
        prob, U = problem_from(w)
        err = rel_linf(b.get_state(i, "cpu"), ro.run(U, prob, 4), w["gamma"])
        assert max(err) < 1e-5, (i, w["n"], err)
    b.close()


def test_mixed_batch_with_and_without_background():
    """One batch holding runs with a y background and runs without one
    (plain float32 storage, periodic and walled), each against the oracle."""
    ws = small_batch(3) + [inputs.random_smooth_state(2, (50, 34), xi=5.0, variant="pms"),
                           inputs.random_smooth_state(2, (72, 40), xi=2.0, variant="dvs",
                                                      bc=("reflect", "periodic"), grav=(0.3, 0.0, 0.0))]
    b = rsst.BatchSolver(ws)
    for i, w in enumerate(ws):
        b.set_state(i, torch.from_numpy(w["U"]).cuda())
    b.step(4)
    b.sync()
    for i, w in enumerate(ws):
        prob, U = problem_from(w)
        err = rel_linf(b.get_state(i, "cpu"), ro.run(U, prob, 4), w["gamma"])
        assert max(err) < 1e-5, (i, w["n"], w["vertical"], err)
    b.close()
