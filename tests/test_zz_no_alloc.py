"""The allocation-free conservation sums against the handle-based ones.

Some callers cannot allocate device memory at the moment they need the sums
(for instance inside another framework that owns the device-memory
budget).  rsst_conserved_sums_noalloc serves
them with a fixed device-side scratch array; here it must agree with
rsst_conserved_sums on the same states, on two calls in a row.  Both use the
same fixed reduction tree (1024 contiguous chunks, the same thread striding
and shared-memory tree, the partials summed in index order, then one
multiplication by the cell volume), so the results must be equal bit for
bit.  This file is collected last so that a failure here never hides another
test."""
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


def _handle_sums(w):
    s = rsst.Solver(w, "fp64")
    s.set_state(torch.from_numpy(w["U"]).cuda())
    out = s.sums()
    s.close()
    return out


@pytest.mark.parametrize("ndim,n", [(1, (300,)), (2, (70, 37)), (3, (35, 18, 11))])
def test_noalloc_sums_match_handle_sums_twice(ndim, n):
    states = [inputs.random_smooth_state(ndim, n, xi=3.0, seed=31),
              inputs.random_smooth_state(ndim, n, xi=3.0, seed=47)]
    for w in states:                         # two calls in a row, different inputs
        want = _handle_sums(w)
        U = torch.from_numpy(w["U"]).cuda()
        got = torch.full((ndim + 2,), float("nan"), dtype=torch.float64, device="cuda")
        rsst.rsst_conserved_sums_noalloc(U, w["n"], w["dx"], got)
        torch.cuda.synchronize()
        assert got.tolist() == want, (got.tolist(), want)


def test_noalloc_rejects_oversized_input():
    U = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = torch.zeros(6, dtype=torch.float64, device="cuda")
    with pytest.raises(rsst.RsstError) as e:
        rsst.rsst_conserved_sums_noalloc(U, (1, 1, 1, 1), (1.0,) * 4, out)
    assert e.value.code == rsst.RSST_EINVAL
    with pytest.raises(rsst.RsstError) as e:
        rsst.rsst_conserved_sums_noalloc(U, (1 << 16, 1 << 16), (1.0, 1.0), out)
    assert e.value.code == rsst.RSST_EINVAL
