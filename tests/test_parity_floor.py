"""The round-off floor the float64 parity tests fall back on (tests/parity.py),
checked on the CPU: it leaves the oracle untouched, it is reproducible, it is
round-off sized on a well-conditioned run, it rises where a field's own size
is at the round-off level of the terms that produce it, and it does not
excuse a real deviation."""
import pytest
import torch

from oracle import rsst_oracle as ro
from oracle.workload import problem_from
from paper_1812_04135_gb300 import inputs
from tests.parity import FLOOR_FACTOR, assert_parity, roundoff_floor


def _case():
    w = inputs.random_smooth_state(2, (24, 20), xi=4.0, variant="pvs")
    prob, U = problem_from(w)
    return w, prob, U, ro.run(U, prob, 4)


def test_floor_leaves_the_oracle_untouched_and_is_reproducible():
    w, prob, U, ref = _case()
    f1 = roundoff_floor(U, prob, 4, ref, w)
    f2 = roundoff_floor(U, prob, 4, ref, w)
    assert f1 == f2
    assert torch.equal(ro.run(U, prob, 4), ref)   # the wrapped entry points were restored
    assert max(f1) > 0.0                           # the perturbation was applied
    assert max(f1) < 1e-13                         # and it is round-off sized here


def test_floor_rises_where_a_field_is_round_off_of_larger_terms():
    """The 1D sound eigenmode at xi = 10 with amplitude 1e-6: its momentum is
    1e-5 of the pressure flux that drives it, so after 200 steps round-off
    of that flux is ~1e-9 of the momentum itself."""
    w = inputs.sound_wave_1d(256, xi=10.0, variant="pvs")
    prob, U = problem_from(w)
    ref = ro.run(U, prob, 200)
    f = roundoff_floor(U, prob, 200, ref, w)
    assert f[1] > 1e-11 and f[0] < 1e-13, f


def test_assert_parity_rejects_a_real_deviation_and_accepts_round_off():
    w, prob, U, ref = _case()
    bumped = ref.clone()
    bumped[1] = bumped[1] * (1.0 + 1e-8)           # a real deviation of the momentum
    with pytest.raises(AssertionError):
        assert_parity(bumped, ref, w, U, prob, 4)
    ulp = ref.clone()
    ulp[0] = torch.nextafter(ulp[0], torch.full_like(ulp[0], 10.0))  # one ulp of rho
    assert max(assert_parity(ulp, ref, w, U, prob, 4)) < 1e-10
    assert FLOOR_FACTOR <= 8.0
