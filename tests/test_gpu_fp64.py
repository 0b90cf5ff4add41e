"""Float64 CUDA path vs the CPU oracle, element by element, through the C ABI.

Tolerance: relative L-infinity 1e-10 per field (tests/parity.py).  Sizes
span several tiles with ragged tails on every axis; all forms, both wall
types, gravity with a background, and the workloads' full sizes."""
import math

import numpy as np
import pytest
import torch

from oracle import rsst_oracle as ro
from oracle.workload import problem_from
from paper_1812_04135_gb300 import inputs, rsst
from tests.parity import assert_parity

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import os
    if not os.path.exists(rsst.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    rsst.lib()
    torch.cuda.init()


def gpu_run(w, nsteps, dt=0.0, precision="fp64", **over):
    s = rsst.Solver(w, precision, **over)
    try:
        s.set_state(torch.from_numpy(w["U"]).cuda())
        s.step(nsteps, dt)
        return s.get_state("cpu")
    finally:
        s.close()


def check(w, nsteps, dt=0.0, tol=TOL, what=""):
    """GPU run vs the oracle run on the same input: every field within 1e-10
    of its own size, or, where a few ulps of the full field already exceed
    that, within the oracle's own round-off floor (tests/parity.py)."""
    prob, U = problem_from(w)
    odt = dt if dt > 0.0 else None
    ref = ro.run(U, prob, nsteps, dt=odt)
    assert_parity(gpu_run(w, nsteps, dt), ref, w, U, prob, nsteps, dt=odt, precision="fp64", tol=tol, what=what)


SIZES = {1: (300,), 2: (70, 37), 3: (35, 18, 11)}


@pytest.mark.parametrize("ndim", [1, 2, 3])
@pytest.mark.parametrize("var", ["euler", "dvs", "pvs", "dms", "pms", "pd"])
def test_periodic_all_forms(ndim, var):
    w = inputs.random_smooth_state(ndim, SIZES[ndim], xi=6.0, variant=var)
    check(w, 4, what=(ndim, var))


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_reflecting_walls_and_gravity(ndim):
    bc = ("reflect", "periodic", "reflect")[:ndim] if ndim > 1 else ("reflect",)
    grav = (0.3, -0.8, 0.5)[:ndim] + (0.0,) * (3 - ndim)
    for var in ("pvs", "dms"):
        w = inputs.random_smooth_state(ndim, SIZES[ndim], xi=5.0, variant=var, bc=bc, grav=grav)
        check(w, 4, what=(ndim, var))


def test_stratified_background_2d():
    w = inputs.polytrope_2d(40, 70, xi=20.0, contrast=20.0, amp=1e-2)
    for var in ("pvs", "pms", "dvs"):
        w["variant"] = var
        check(w, 6, what=var)


def test_stratified_background_3d_small():
    w = inputs.polytrope_3d(20, 12, 40, xi=50.0, amp=1e-2, contrast=20.0)
    check(w, 5)


def test_fixed_dt_and_many_steps():
    w = inputs.random_smooth_state(2, (40, 34), xi=4.0, variant="pms")
    check(w, 20, dt=1e-3)
    check(w, 50)


def test_dt_matches_cfl_rule():
    w = inputs.shear_layer_2d(64, 48, xi=30.0)
    s = rsst.Solver(w, "fp64")
    s.set_state(torch.from_numpy(w["U"]).cuda())
    prob, U = problem_from(w)
    assert s.dt() == pytest.approx(ro.cfl_dt(U, prob), rel=1e-13)
    s.step(3)
    U3 = ro.run(U, prob, 3)
    assert s.dt() == pytest.approx(ro.cfl_dt(U3, prob), rel=1e-12)
    s.close()


def test_sound_wave_workload_1d():
    """1D N = 256 sound eigenmode at xi = 10, 200 steps (a/xi travel)."""
    for xi, var in ((10.0, "pvs"), (1.0, "dvs"), (10.0, "pms")):
        w = inputs.sound_wave_1d(256, xi=xi, variant=var)
        check(w, 200, what=(xi, var))


def test_contact_workload_1d():
    for xi, var in ((10.0, "pvs"), (1.0, "dvs"), (10.0, "pd")):
        w = inputs.contact_1d(256, xi=xi, variant=var)
        check(w, 10, what=(xi, var))


def test_shear_layer_full_size():
    """2D 512 x 512 shear layer, xi = 30, full-grid comparison."""
    w = inputs.shear_layer_2d()
    for var in ("pvs", "dvs"):
        w["variant"] = var
        check(w, 3, what=var)


def test_polytrope_full_size_one_step():
    """3D 256 x 128 x 128 stratified box, xi = 50, one step on the full grid."""
    w = inputs.polytrope_3d()
    check(w, 1)


def test_momentum_conserved_to_round_off():
    w = inputs.shear_layer_2d(256, 256, xi=30.0, variant="pms")
    s = rsst.Solver(w, "fp64")
    s.set_state(torch.from_numpy(w["U"]).cuda())
    s0 = s.sums()
    s.step(200)
    s1 = s.sums()
    U = torch.from_numpy(w["U"])
    scale_m = float((U[1].abs().sum() + U[2].abs().sum())) / (256 * 256)
    for k in (1, 2):
        assert abs(s1[k] - s0[k]) < 1e-13 * scale_m * 200, (k, s0[k], s1[k])
    assert abs(s1[0] - s0[0]) > 0          # PMS carries a mass source
    s.close()


def test_mass_conserved_dms():
    w = inputs.shear_layer_2d(256, 128, xi=30.0, variant="dms")
    s = rsst.Solver(w, "fp64")
    s.set_state(torch.from_numpy(w["U"]).cuda())
    s0 = s.sums()
    s.step(200)
    s1 = s.sums()
    assert abs(s1[0] - s0[0]) < 1e-13 * abs(s0[0]) * 10
    s.close()


def test_sums_match_exact_sums():
    w = inputs.random_smooth_state(3, (33, 17, 9), xi=3.0)
    s = rsst.Solver(w, "fp64")
    s.set_state(torch.from_numpy(w["U"]).cuda())
    got = s.sums()
    prob, U = problem_from(w)
    want = ro.conserved_sums(U, prob)
    for g, e, k in zip(got, want, range(5)):
        assert g == pytest.approx(e, rel=1e-13, abs=1e-15), k
    s.close()


def test_nonphysical_state_is_flagged():
    """The ratio-10 contact cannot run the density-reduced form at xi = 10
    (Sec. 2.2): the step must report RSST_ENONPHYSICAL, not crash."""
    w = inputs.contact_1d(256, xi=10.0, variant="dvs")
    s = rsst.Solver(w, "fp64")
    s.set_state(torch.from_numpy(w["U"]).cuda())
    s.step(3)
    with pytest.raises(rsst.RsstError) as e:
        s.sync()
    assert e.value.code == rsst.RSST_ENONPHYSICAL
    # a fresh state clears the flag
    w2 = inputs.contact_1d(256, xi=10.0, variant="pvs")
    s.set_state(torch.from_numpy(w2["U"]).cuda())
    s.sync()
    s.close()


def test_host_buffers_roundtrip():
    w = inputs.random_smooth_state(2, (50, 20), xi=3.0)
    s = rsst.Solver(w, "fp64")
    s.set_state(torch.from_numpy(w["U"]).pin_memory())
    got = s.get_state("cpu")
    assert torch.equal(got, torch.from_numpy(w["U"]))
    s.close()


def test_float64_helpers_against_cuda():
    """Newton-Raphson reciprocal within 1 ulp of CUDA's 1.0/x; integer-pipe
    MC limiter identical to the direct float64 form; the c_tot square root
    within 2^-40 of CUDA's sqrt, with its special cases."""
    ulp, bad, rel = rsst.rsst_math_selftest(1 << 20)
    assert ulp <= 1.0 and bad == 0, (ulp, bad)
    assert rel <= 2.0 ** -40, rel


def test_fp64_fma_peak_probe():
    """The float64 throughput probe behind the arithmetic roofline returns a
    plausible rate (GB300: about 1.2 TFLOP/s)."""
    tf, ms = rsst.rsst_fp64_fma_peak(2000)
    assert 0.2 < tf < 5.0 and ms > 0.0, (tf, ms)


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_cmax_law(ndim):
    """State-dependent xi = [1 + (a/C_max)^4]^(1/4) (Eq. cx) in c_tot and f."""
    for var, bc, grav in (("pvs", None, (0.0, 0.0, 0.0)), ("dms", ("reflect",) * ndim, (0.2, -0.5, 0.3))):
        w = inputs.random_smooth_state(ndim, SIZES[ndim], xi=1.0, variant=var, bc=bc, grav=grav)
        w["cmax"] = 0.35
        check(w, 4, what=(ndim, var))


def test_cmax_stratified_background():
    w = inputs.polytrope_2d(40, 70, xi=1.0, contrast=20.0, amp=1e-2)
    w["cmax"] = 0.05
    check(w, 6)


@pytest.mark.parametrize("n", [19456, 19457, 20011])
def test_long_1d_lines_use_wide_tiles(n):
    """Lines up to 32*152*4 cells run in 32-cell tiles, longer ones in
    256-cell tiles: both shapes, and the boundary between them, match."""
    w = inputs.random_smooth_state(1, (n,), xi=6.0, variant="pvs", bc=("reflect",), grav=(0.5, 0.0, 0.0))
    check(w, 3, what=n)


def test_c_abi_rejects_the_wrong_kind_of_buffer():
    """The C ABI itself (below the binding's checks) refuses a host buffer
    passed as device memory and a device buffer passed as host memory, with
    RSST_EINVAL and before any copy or kernel runs.  The host buffer is
    pinned, so even a missed check could not make the GPU fault."""
    w = inputs.random_smooth_state(2, (16, 12), xi=3.0)
    s = rsst.Solver(w, "fp64")
    L = rsst.lib()
    host = torch.from_numpy(w["U"]).pin_memory()
    dev = torch.from_numpy(w["U"]).cuda()
    assert L.rsst_set_state(s.h, host.data_ptr(), 0) == rsst.RSST_EINVAL
    assert b"host memory" in L.rsst_last_error()
    assert L.rsst_get_state(s.h, dev.data_ptr(), 1) == rsst.RSST_EINVAL
    assert L.rsst_set_state(s.h, dev.data_ptr(), 0) == rsst.RSST_OK
    assert L.rsst_get_state(s.h, host.data_ptr(), 1) == rsst.RSST_OK
    assert torch.equal(host, torch.from_numpy(w["U"]))
    s.close()


def test_shear_layer_512_conservation_by_form():
    """The 512 x 512 shear layer at xi = 30 (density ratio 10, Mach 0.01), by
    form: PMS holds total momentum to round-off over 5000 steps (bound
    10 x steps x eps x sum|m|) while its mass source moves the mass; DMS holds
    mass and momentum to round-off while it stays physical; the
    density-reduced forms DVS and DMS become non-physical at the ratio-10
    interface within 5000 steps (the drawback of Sec. 2.2), reported as
    RSST_ENONPHYSICAL."""
    eps = 2.2e-16
    w = inputs.shear_layer_2d(512, 512, xi=30.0, variant="pms")
    U = torch.from_numpy(w["U"])
    vol = 1.0 / (512 * 512)
    absq = [float(U[k].abs().sum()) * vol for k in range(4)]
    s = rsst.Solver(w, "fp64")
    s.set_state(U.cuda())
    s0 = s.sums()
    s.step(5000)
    s1 = s.sums()
    s.close()
    for k in (1, 2):
        assert abs(s1[k] - s0[k]) <= 10 * 5000 * eps * absq[k], (k, s0[k], s1[k])
    assert abs(s1[0] - s0[0]) > 1e-9 * absq[0]                      # PMS carries a mass source
    w["variant"] = "dms"
    s = rsst.Solver(w, "fp64")
    s.set_state(U.cuda())
    s0 = s.sums()
    s.step(200)
    s1 = s.sums()
    s.close()
    for k in (0, 1, 2):
        assert abs(s1[k] - s0[k]) <= 10 * 200 * eps * absq[k], (k, s0[k], s1[k])
    for var in ("dvs", "dms"):
        w["variant"] = var
        s = rsst.Solver(w, "fp64")
        s.set_state(U.cuda())
        with pytest.raises(rsst.RsstError) as e:
            for _ in range(50):
                s.step(100)
                s.sync()
        assert e.value.code == rsst.RSST_ENONPHYSICAL, var
        s.close()


def _gpu_phase_speed(w, nsteps, every, field):
    """Phase speed of Fourier mode 1 of P or rho from GPU snapshots every
    ``every`` steps, with the device's simulated time."""
    s = rsst.Solver(w, "fp64")
    s.set_state(torch.from_numpy(w["U"]).cuda())
    ts, ph = [], []
    for k in range(nsteps // every + 1):
        if k:
            s.step(every)
        U = s.get_state("cpu").numpy()
        rho, m, E = U[0], U[1], U[2]
        q = (w["gamma"] - 1.0) * (E - 0.5 * m * m / rho) if field == "P" else rho
        ts.append(s.time())
        ph.append(float(np.angle(np.fft.rfft(q - q.mean())[1])))
    s.close()
    slope = np.polyfit(np.array(ts), np.unwrap(np.array(ph)), 1)[0]
    return -slope / (2 * math.pi)


@pytest.mark.parametrize("var,xi", [("pvs", 10.0), ("dvs", 10.0), ("pvs", 1.0), ("dvs", 1.0), ("pms", 10.0)])
def test_sound_wave_speed_2000_steps(var, xi):
    """1D N = 256 sound eigenmode, 2000 steps on the GPU: it travels at a/xi
    (a = 1 here) within 1 % (Sec. 3.1)."""
    w = inputs.sound_wave_1d(256, xi=xi, variant=var)
    assert _gpu_phase_speed(w, 2000, 50, "P") == pytest.approx(1.0 / xi, rel=0.01)


@pytest.mark.parametrize("var,xi", [("pvs", 10.0), ("pms", 10.0), ("dvs", 1.0)])
def test_entropy_wave_keeps_flow_speed_2000_steps(var, xi):
    """The density-10 contact keeps the flow speed u = 0.01 within 2 % over
    2000 steps on the GPU (the entropy wave is not slowed by xi)."""
    w = inputs.contact_1d(256, xi=xi, variant=var)
    assert _gpu_phase_speed(w, 2000, 100, "rho") == pytest.approx(0.01, rel=0.02)
