"""The C-ABI library loads without a GPU, exports every function declared in
include/*.h, matches the binding's struct layout, and rejects invalid
configurations before touching the device."""
import glob
import os
import re

import pytest

from paper_1812_04135_gb300 import rsst

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(rsst_\w+)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(rsst.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return rsst.lib()


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert len(names) >= 10
    for n in sorted(names):
        assert hasattr(L, n), n


def test_config_layout(L):
    assert L.rsst_config_size() == 144


@pytest.mark.parametrize("bad", [dict(ndim=4), dict(xi=0.5), dict(gamma=1.0), dict(variant="bogus"),
                                 dict(n0=1), dict(cfl=0.0), dict(vertical=1)])
def test_invalid_config_rejected_without_gpu(L, bad):
    kw = dict(variant="pvs", xi=3.0)
    ndim, n = 2, [8, 8, 1]
    if "ndim" in bad:
        ndim = bad["ndim"]
    if "n0" in bad:
        n[0] = bad["n0"]
    for k in ("xi", "gamma", "cfl", "vertical"):
        if k in bad:
            kw[k] = bad[k]
    if bad.get("variant") == "bogus":
        kw["variant"] = 17
    cfg = rsst.make_config(ndim, n, [0.1, 0.1, 0.1], **kw)
    with pytest.raises(rsst.RsstError) as e:
        rsst.rsst_init(cfg, stream=0)
    assert e.value.code == rsst.RSST_EINVAL


def test_graph_steps_rejects_null_handle_and_odd_k(L):
    assert L.rsst_set_graph_steps(None, 16) == rsst.RSST_EINVAL
    assert L.rsst_set_graph_steps(None, 3) == rsst.RSST_EINVAL


def test_binding_rejects_wrong_buffers_before_the_library():
    """The C ABI takes bare pointers; the binding checks dtype, contiguity and
    where the buffer lives before any call reaches the library."""
    import numpy as np
    import torch
    with pytest.raises(ValueError):
        rsst.rsst_set_state(0, np.zeros(8, dtype=np.float32), on_host=True)
    with pytest.raises(ValueError):
        rsst.rsst_set_state(0, np.zeros(8), on_host=False)          # host array passed as device memory
    with pytest.raises(ValueError):
        rsst.rsst_get_state(0, torch.zeros(8, dtype=torch.float64), on_host=False)
    with pytest.raises(ValueError):
        rsst.rsst_set_state(0, torch.zeros(4, 4, dtype=torch.float64).t(), on_host=True)  # not contiguous
    with pytest.raises(ValueError):
        rsst.rsst_adjoint_step(0, 0, torch.zeros(8, dtype=torch.float64))                 # must be a CUDA tensor
