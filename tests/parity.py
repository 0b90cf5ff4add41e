"""Parity helpers shared by the GPU tests (test infrastructure).

Two per-field relative L-infinity errors, max_cells |gpu - ref| over a scale:

- ``rel_linf_own`` (the float64 bar): each field over its own size.  rho and
  E over max |ref - U0|, U0 the workload's hydrostatic background (zero
  without one), so a stratified run is judged on its perturbation; each
  momentum component over max |m_ref| (over rho (|V| + a) only where the
  reference momentum is exactly zero).  In the low-Mach workloads the
  momentum is far smaller than rho times the sound speed, so this is the
  strict scale.
- ``rel_linf`` (the float32 bar): rho and E over max |ref|, momentum over
  max rho (|V| + a), the field scale the float32 tolerance is stated on; the
  float32 tests add ``rel_linf_pert`` on stratified runs.

Where a field's own size is so small that a few units in the last place of
the full field already exceed 1e-10 of it (a density perturbation of 1e-5
on rho ~ 10, momentum that is zero by symmetry and holds only round-off, a
low-Mach momentum beside a P = 1000 pressure flux), no float64 program that
rounds differently from the oracle can meet 1e-10 on that scale.
``assert_parity`` then measures the problem's own round-off floor: the
oracle is run again with every face flux and every tendency multiplied by
(1 + r), r uniform in [-u, u] (seeded; u the unit round-off of the
precision), and so is the state each stage reads (the rounding of the stored
state), and the per-field difference from the plain oracle run is the
floor.  The GPU result passes a field if its error is below 1e-10 or below
FLOOR_FACTOR times that floor.  Both numbers are logged.

With RSST_PARITY_LOG set to a file name, every ``rel_linf_own`` call and
every ``assert_parity`` call appends a JSON line (test id, errors, floor) to
it, so a run records the measured values."""
import contextlib
import json
import os

import numpy as np
import torch


def field_scales(ref: torch.Tensor, gamma: float):
    ref = ref.double().cpu()
    nd = ref.shape[0] - 2
    rho = ref[0]
    v2 = sum((ref[1 + d] / rho) ** 2 for d in range(nd))
    P = (gamma - 1.0) * (ref[-1] - 0.5 * rho * v2)
    a = torch.sqrt(torch.clamp(gamma * P / rho, min=0.0))
    mscale = float((rho * (torch.sqrt(v2) + a)).max())
    return [float(ref[0].abs().max())] + [mscale] * nd + [float(ref[-1].abs().max())]


def rel_linf(got: torch.Tensor, ref: torch.Tensor, gamma: float):
    got = got.double().cpu()
    ref = ref.double().cpu()
    sc = field_scales(ref, gamma)
    return [float((got[k] - ref[k]).abs().max()) / sc[k] for k in range(ref.shape[0])]


_ORACLE_CACHE = {}


def oracle_cached(key, fn):
    """Memoise an expensive oracle result within one test process."""
    if key not in _ORACLE_CACHE:
        _ORACLE_CACHE[key] = fn()
    return _ORACLE_CACHE[key]


def background_state(w) -> torch.Tensor:
    """U0 = (rho0, 0, P0/(gamma-1)) of a workload's background, broadcast to its grid."""
    nd = w["ndim"]
    shape = tuple(reversed(w["n"]))
    U0 = torch.zeros((nd + 2,) + shape, dtype=torch.float64)
    if w["bg_rho"] is None:
        return U0
    v = w["vertical"]
    nv = w["n"][v]
    r0 = torch.as_tensor(w["bg_rho"][2:2 + nv], dtype=torch.float64)
    e0 = torch.as_tensor(w["bg_p"][2:2 + nv], dtype=torch.float64) / (w["gamma"] - 1.0)
    ax = nd - 1 - v
    view = [1] * nd
    view[ax] = nv
    U0[0] = r0.reshape(view).expand(shape)
    U0[-1] = e0.reshape(view).expand(shape)
    return U0


def rel_linf_pert(got, ref, w):
    """Per-field max |gpu - ref| over max |ref - U0|: the error relative to the
    perturbation about the background (what the float32 mode must keep)."""
    U0 = background_state(w)
    got = got.double().cpu()
    ref = ref.double().cpu()
    out = []
    for k in range(ref.shape[0]):
        den = float((ref[k] - U0[k]).abs().max())
        num = float((got[k] - ref[k]).abs().max())
        out.append(num / den if den > 0 else (0.0 if num == 0.0 else float("inf")))
    return out


def permute(w, order):
    """Relabel the axes of a workload: new axis d is old axis order[d]."""
    nd = w["ndim"]
    U = w["U"]                                     # [nvar][z][y][x] (reversed axes)
    # tensor axis of grid axis d is 1 + (nd - 1 - d)
    perm = [0] + [1 + (nd - 1 - order[nd - 1 - t]) for t in range(nd)]
    V = np.ascontiguousarray(np.transpose(U, perm))
    mom = [V[1 + order[d]] for d in range(nd)]     # momentum components follow their axes
    V = np.ascontiguousarray(np.stack([V[0]] + mom + [V[nd + 1]]))
    out = dict(w)
    out["U"] = V
    out["n"] = tuple(w["n"][order[d]] for d in range(nd))
    out["dx"] = tuple(w["dx"][order[d]] for d in range(nd))
    out["bc"] = tuple(w["bc"][order[d]] for d in range(nd))
    out["grav"] = tuple(w["grav"][order[d]] for d in range(nd)) + (0.0,) * (3 - nd)
    out["vertical"] = order.index(w["vertical"])
    return out


def column_1d(w2):
    """The vertical column x = 0 of a 2D stratified workload as a 1D run along x."""
    U = w2["U"][:, :, 0]                           # [rho, m_x, m_y, E] along y
    V = np.ascontiguousarray(np.stack([U[0], U[2], U[3]]))
    out = dict(w2)
    out.update(ndim=1, U=V, n=(w2["n"][1],), dx=(w2["dx"][1],), bc=(w2["bc"][1],),
               grav=(w2["grav"][1], 0.0, 0.0), vertical=0)
    return out


def own_scales(ref: torch.Tensor, w):
    """Each field's own scale (see the module docstring)."""
    ref = ref.double().cpu()
    nd = ref.shape[0] - 2
    U0 = background_state(w) if w.get("bg_rho") is not None else torch.zeros_like(ref)
    fallback = field_scales(ref, w["gamma"])
    out = []
    for k in range(ref.shape[0]):
        if 1 <= k <= nd:
            den = float(ref[k].abs().max())
        else:
            den = float((ref[k] - U0[k]).abs().max())
        out.append(den if den > 0.0 else fallback[k])
    return out


def _own_err(got: torch.Tensor, ref: torch.Tensor, w):
    got = got.double().cpu()
    ref = ref.double().cpu()
    sc = own_scales(ref, w)
    return [float((got[k] - ref[k]).abs().max()) / sc[k] for k in range(ref.shape[0])]


def _log(rec):
    log = os.environ.get("RSST_PARITY_LOG")
    if log:
        rec = dict(test=os.environ.get("PYTEST_CURRENT_TEST", ""), **rec)
        with open(log, "a") as f:
            f.write(json.dumps(rec) + "\n")


def rel_linf_own(got: torch.Tensor, ref: torch.Tensor, w):
    """Per-field max |gpu - ref| over the field's own scale (own_scales)."""
    err = _own_err(got, ref, w)
    _log({"err": err})
    return err


# float64: 2^-53.  Double-float stores 24 + 24 significant bits (2^-48), and its
# product and quotient sequences are accurate to about 5 units of that
# (Joldes, Muller and Popescu 2017, double-word arithmetic error bounds).
UNIT_ROUNDOFF = {"fp64": 2.0 ** -53, "fp64_df": 5.0 * 2.0 ** -48}
FLOOR_FACTOR = 4.0


@contextlib.contextmanager
def _rounding_perturbed_oracle(unit: float, seed: int):
    """The oracle with every face flux, every tendency and the state every
    tendency reads multiplied by (1 + r), r uniform in [-unit, unit] from a
    seeded generator.  Only the
    module's entry points are wrapped (restored on exit); its arithmetic is
    untouched."""
    from oracle import rsst_oracle as ro
    g = torch.Generator().manual_seed(seed)

    def jitter(x):
        return x * (1.0 + (torch.rand(x.shape, generator=g, dtype=torch.float64) * 2.0 - 1.0) * unit)

    face_fluxes, rhs = ro.face_fluxes, ro.rhs
    ro.face_fluxes = lambda U, d, prob: jitter(face_fluxes(U, d, prob))
    # the stage input is jittered too: the rounding of the stored state (U^n, U*)
    ro.rhs = lambda U, prob: jitter(rhs(jitter(U), prob))
    try:
        yield ro
    finally:
        ro.face_fluxes, ro.rhs = face_fluxes, rhs


def roundoff_floor(U, prob, nsteps, ref, w, dt=None, unit=2.0 ** -53, seed=0):
    """Per-field own-scale difference between the oracle run (ref) and the
    same run with round-off-sized perturbations (see the module docstring)."""
    with _rounding_perturbed_oracle(unit, seed) as ro:
        alt = ro.run(U, prob, nsteps, dt=dt)
    return _own_err(alt, ref, w)


def assert_parity(got, ref, w, U, prob, nsteps, dt=None, precision="fp64", tol=1e-10, what=""):
    """GPU result vs the oracle's: every field's own-scale error below tol, or,
    for a field where that is below the representation's reach, below
    FLOOR_FACTOR times the oracle's own round-off floor on the same run."""
    err = _own_err(got, ref, w)
    floor = None
    if max(err) >= tol:
        floor = roundoff_floor(U, prob, nsteps, ref, w, dt=dt, unit=UNIT_ROUNDOFF[precision])
    _log({"err": err, "floor": floor, "precision": precision, "nsteps": nsteps})
    bound = [max(tol, FLOOR_FACTOR * f) for f in floor] if floor else [tol] * len(err)
    assert all(e < b for e, b in zip(err, bound)), (what, "err", err, "floor", floor)
    return err


def check_precision(got, ref, w, U, prob, nsteps, precision: str, tol: float, dt=None, what=""):
    """The bar of each precision: assert_parity (own scales, round-off floor)
    for float64 and double-float, the field scale for the float32
    perturbation mode."""
    if precision == "fp32_pert":
        err = rel_linf(got, ref, w["gamma"])
        assert max(err) < tol, (what, err)
        return err
    return assert_parity(got, ref, w, U, prob, nsteps, dt=dt, precision=precision, tol=tol, what=what)
