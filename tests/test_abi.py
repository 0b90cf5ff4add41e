"""The C-ABI library loads without a GPU, exports every function declared in
include/*.h, matches the binding's struct layout, and rejects invalid
configurations before touching the device."""
import glob
import os
import re

import numpy as np
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
    assert L.rsst_config_size() == 152


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


@pytest.mark.parametrize("cov,precision,code", [(-0.1, "fp64", "RSST_EINVAL"), (float("nan"), "fp64", "RSST_EINVAL"),
                                                (0.1, "fp32_pert", "RSST_EUNSUPPORTED"),
                                                (0.1, "fp64_df", "RSST_EUNSUPPORTED")])
def test_covolume_checked_without_gpu(L, cov, precision, code):
    """The covolume gas: b >= 0 and finite, and only in the float64 precision."""
    cfg = rsst.make_config(2, [8, 8, 1], [0.1, 0.1, 0.1], xi=3.0, precision=precision, covolume=cov)
    with pytest.raises(rsst.RsstError) as e:
        rsst.rsst_init(cfg, stream=0)
    assert e.value.code == getattr(rsst, code)


def test_background_beyond_the_covolume_rejected_without_gpu(L):
    """A background density with b rho0 >= 1 is outside the covolume gas."""
    rho, p = np.linspace(2.0, 1.0, 12), np.linspace(3.0, 1.0, 12)
    cfg = rsst.make_config(2, [6, 8, 1], [0.1, 0.1, 0.1], xi=3.0, bc=("periodic", "reflect"), vertical=1,
                           bg_rho=rho, bg_p=p, covolume=0.5)
    with pytest.raises(rsst.RsstError) as e:
        rsst.rsst_init(cfg, stream=0)
    assert e.value.code == rsst.RSST_EINVAL and "covolume" in str(e.value)


@pytest.mark.parametrize("bc,k,field,value", [("reflect", 0, "rho", -1.0), ("reflect", 11, "p", 0.0),
                                               ("periodic", 5, "rho", float("nan")), ("reflect", 3, "p", float("inf"))])
def test_bad_background_rejected_without_gpu(L, bc, k, field, value):
    """rsst_init reads every background entry it uses (all n + 4 on a wall
    axis, the interior on a periodic one) and rejects a non-physical one
    before any device call."""
    rho, p = np.linspace(2.0, 1.0, 12), np.linspace(3.0, 1.0, 12)
    (rho if field == "rho" else p)[k] = value
    cfg = rsst.make_config(2, [6, 8, 1], [0.1, 0.1, 0.1], xi=3.0, bc=("periodic", bc), vertical=1, bg_rho=rho, bg_p=p)
    with pytest.raises(rsst.RsstError) as e:
        rsst.rsst_init(cfg, stream=0)
    assert e.value.code == rsst.RSST_EINVAL
    assert "background" in str(e.value)


def test_periodic_background_ghost_entries_are_not_read(L):
    """On a periodic vertical axis the ghost entries are taken by wrap, so a
    NaN there passes validation (the call then fails only at the device)."""
    rho, p = np.linspace(2.0, 1.0, 12), np.linspace(3.0, 1.0, 12)
    rho[0] = rho[-1] = float("nan")
    cfg = rsst.make_config(2, [6, 8, 1], [0.1, 0.1, 0.1], xi=3.0, bc=("periodic", "periodic"), vertical=1,
                           bg_rho=rho, bg_p=p)
    try:
        h = rsst.rsst_init(cfg, stream=0)
    except rsst.RsstError as e:
        assert "background" not in str(e), str(e)
    else:
        rsst.rsst_destroy(h)


@pytest.mark.parametrize("field,value", [("grav", float("inf")), ("gamma", float("inf")), ("cfl", float("nan")),
                                         ("cfl_rule", 2), ("cfl_rule", -1)])
def test_non_finite_parameters_rejected_without_gpu(L, field, value):
    kw = dict(variant="pvs", xi=3.0)
    kw[field] = (0.0, value, 0.0) if field == "grav" else value
    cfg = rsst.make_config(2, [8, 8, 1], [0.1, 0.1, 0.1], **kw)
    with pytest.raises(rsst.RsstError) as e:
        rsst.rsst_init(cfg, stream=0)
    assert e.value.code == rsst.RSST_EINVAL


def test_binding_checks_background_length():
    with pytest.raises(ValueError):
        rsst.make_config(2, [6, 8, 1], [0.1] * 3, vertical=1, bg_rho=np.ones(8), bg_p=np.ones(8))


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


def test_rho_fixed_vp_rejects_bad_arguments_without_gpu(L):
    import ctypes as C
    import torch
    n = (C.c_int32 * 2)(4, 3)
    assert L.rsst_adjoint_rho_fixed_vp(None, None, None, 2, n, None) == rsst.RSST_EINVAL
    assert L.rsst_adjoint_rho_fixed_vp(None, None, None, 4, n, None) == rsst.RSST_EINVAL
    with pytest.raises(ValueError):   # host tensors
        rsst.rsst_adjoint_rho_fixed_vp(torch.zeros(4, 3, 4, dtype=torch.float64), torch.zeros(4, 3, 4, dtype=torch.float64),
                                       torch.zeros(3, 4, dtype=torch.float64))
    with pytest.raises(ValueError):   # shape mismatch
        rsst.rsst_adjoint_rho_fixed_vp(torch.zeros(4, 3, 4, dtype=torch.float64), torch.zeros(4, 3, 5, dtype=torch.float64),
                                       torch.zeros(3, 4, dtype=torch.float64))


def test_header_is_plain_c_and_matches_the_library(L, tmp_path):
    """include/rsst.h compiles as strict C99 (the boundary is a C ABI: plain
    pointers, sizes and enums), and a C program sees the same rsst_config
    size as the library."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_header.c"
    src.write_text('#include <stdio.h>\n#include "rsst.h"\n'
                   'int main(void) { printf("%zu\\n", sizeof(rsst_config)); return 0; }\n')
    exe = tmp_path / "use_header"
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    assert int(out) == L.rsst_config_size()


def test_every_entry_point_cites_its_passage_or_says_it_has_none():
    """Each declaration in include/*.h has its own comment, and that comment
    cites the paper (Sec., Eq., App.) or states that the paper has no
    counterpart (or refers to a documented sibling)."""
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(rsst_\w+)\s*\(", txt, flags=re.M):
            before = txt[:m.start()]
            end = before.rfind("*/")
            assert end >= 0 and before[end + 2:].strip() == "", f"{m.group(1)}: no comment of its own"
            comment = re.sub(r"\s*\n\s*\*?\s*", " ", before[before.rfind("/*", 0, end):end])
            assert re.search(r"Sec\.|Eq\.|App\.|no counterpart|paper has no|See rsst_", comment, flags=re.I), m.group(1)


def test_product_path_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """No CPU fallback: with the shared library absent, the binding raises
    before any computation instead of running something else."""
    monkeypatch.setattr(rsst, "LIB_PATH", str(tmp_path / "absent" / "librsst.so"))
    monkeypatch.setattr(rsst, "_lib", None)
    with pytest.raises(ImportError):
        rsst.lib()
    from paper_1812_04135_gb300 import inputs
    w = inputs.random_smooth_state(1, (8,), xi=2.0)
    with pytest.raises(ImportError):
        rsst.Solver(w, "fp64")
    with pytest.raises(ImportError):
        rsst.BatchSolver([inputs.shear_layer_2d(8, 8)])
    with pytest.raises(ImportError):
        rsst.rsst_init(rsst.config_from_workload(w), stream=0)
