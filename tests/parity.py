"""Parity helpers shared by the GPU tests (test infrastructure).

Relative L-infinity error per conserved field: max_cells |gpu - ref| divided
by max_cells |ref| for rho and E, and by max_cells rho (|V| + a) for each
momentum component (the momentum of a gas at rest is 0, so its natural
scale is rho times the signal speed)."""
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
