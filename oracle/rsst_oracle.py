"""Plain FP64 CPU oracle of the RSST explicit finite-volume step.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this
module: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it.  It shares no code with the CUDA library.

It follows Iijima, Hotta & Imada, "Semi-conservative reduced speed of sound
technique for low Mach number flows with large density variations"
(arXiv:1812.04135):

* Euler tendencies dU = -div F (Sec. 3.2, Eq. pvs_dt0),
* the un-reduced pressure tendency dP (Sec. 3.2, Eq. pvs_dt_dpr; ideal gas,
  Eq. pvs_cons_therm: (de/dP)_rho = 1/(gamma-1), (de/drho)_P = 0),
* the RSST correction of the five semi-conservative forms:
  PVS (Sec. 3.2, Eqs. pvs_dt and pvs_cons_rhs), DVS (App. A.1),
  PMS (App. A.2), DMS (App. A.3), PD (App. A.4),
* the external force (App. B): rho*F added to momentum and rho*V.F to
  energy, dP unchanged,
* the numerical method of Sec. 4.2: MUSCL reconstruction of the conservative
  variables with the monotonized-central limiter, local Lax-Friedrichs flux
  with c_tot = |V| + a/xi, second-order SSP Runge-Kutta, CFL number 0.4 with
  c_tot, in the order of the eight implementation steps listed there.

Readings where the paper is silent:
* MC limiter (only named in Sec. 4.2): MC(a, b) = 0 if a*b <= 0, else the
  one of 2a, 2b, (a+b)/2 with the smallest magnitude; ties go to the first
  in that order.
* |V| in c_tot is the full speed (not the face-normal component); the LLF
  speed of a face is max(c_tot(U_L), c_tot(U_R)), ties to U_L.
* Multi-dimensional CFL: dt = C / max_cells sum_d c_tot / dx_d, C = 0.4,
  taken from U^n and used for both stages.
* SSP-RK2 in Shu-Osher form: U* = U + dt L(U); U^{n+1} = U/2 + (U* + dt L(U*))/2.
* The RSST correction uses cell-centre values of the stage state.
* Boundaries: periodic wrap, or a reflecting (free-slip) wall whose two
  ghost cells mirror the interior with the normal momentum negated; with a
  background profile U0 = (rho0, 0, P0/(gamma-1)) along the vertical axis
  the ghost is U0(ghost) + mirror(U - U0)(image).
* Initial data are point values at cell centres.

State layout: a torch float64 tensor of shape [nvar, nz, ny, nx] (3D),
[nvar, ny, nx] (2D) or [nvar, nx] (1D); nvar = 2 + ndim, components
(rho, m_x[, m_y[, m_z]], E).  Dimension index d = 0, 1, 2 is x, y, z.

Parity is pinned by tests/test_oracle_*.py (closed forms, invariants,
the exact Riemann solution, conservation, eigenvalues of the linearised
operator, finite differences for the adjoint).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional, Sequence

import torch

EULER, DVS, PVS, DMS, PMS, PD = 0, 1, 2, 3, 4, 5
VARIANT_NAMES = {EULER: "euler", DVS: "dvs", PVS: "pvs", DMS: "dms", PMS: "pms", PD: "pd"}
PERIODIC, REFLECT = 0, 1

DT = torch.float64


@dataclass
class Problem:
    """Grid, physics and scheme parameters of one run.

    ``n`` and ``dx`` are ordered (x, y, z) and have ``ndim`` entries.
    ``bc[d]`` is PERIODIC or REFLECT for both ends of axis d.
    ``bg_rho`` / ``bg_p`` (optional) are FP64 background profiles along
    ``vertical`` with n[vertical] + 4 entries (two ghost cells each side).
    ``xi`` may be a float or a 0-d float64 tensor (for autograd).
    """

    ndim: int
    n: Sequence[int]
    dx: Sequence[float]
    gamma: float = 5.0 / 3.0
    xi: object = 1.0
    variant: int = PVS
    grav: Sequence[float] = (0.0, 0.0, 0.0)
    bc: Sequence[int] = (PERIODIC, PERIODIC, PERIODIC)
    cfl: float = 0.4
    vertical: int = -1
    bg_rho: Optional[torch.Tensor] = None
    bg_p: Optional[torch.Tensor] = None
    cmax: Optional[float] = None  # C_max law (Eq. cx) instead of a constant xi
    cfl_rule: int = 0  # 0: dt = C / max sum_d c_tot/dx_d;  1: dt = C min_d dx_d / max c_tot (reading 3)

    @property
    def nvar(self) -> int:
        return 2 + self.ndim

    def axis(self, d: int) -> int:
        """Tensor axis (including the leading variable axis) of dimension d."""
        return 1 + (self.ndim - 1 - d)

    def cell_volume(self) -> float:
        return math.prod(float(h) for h in self.dx[: self.ndim])


# ---------------------------------------------------------------------------
# Equation of state (Sec. 3.2: the equations hold for a general EOS P(rho, S);
# Eq. pvs_cons_therm gives the derivatives the pressure tendency needs)
# ---------------------------------------------------------------------------

class IdealGas:
    """e = P/(gamma-1) (e: internal energy per volume), a^2 = gamma P/rho,
    (de/dP)_rho = 1/(gamma-1), (de/drho)_P = 0 (Sec. 3.2)."""

    def __init__(self, gamma: float):
        self.gamma = float(gamma)

    def pressure(self, rho, eint):
        return (self.gamma - 1.0) * eint

    def internal_energy(self, rho, P):
        return P / (self.gamma - 1.0)

    def sound2(self, rho, P):
        return self.gamma * P / rho

    def de_dP(self, rho, P):
        return 1.0 / (self.gamma - 1.0) + 0.0 * P

    def de_drho(self, rho, P):
        return 0.0 * P


def as_eos(g):
    """An EOS object, or the ideal gas of ratio g."""
    return g if hasattr(g, "pressure") else IdealGas(g)


# ---------------------------------------------------------------------------
# Primitive variables (Sec. 2.1, Sec. 3.2: E = e + rho V^2/2)
# ---------------------------------------------------------------------------

def primitives(U: torch.Tensor, gamma):
    """Return rho, list of V_d, |V|^2, P, a^2 of a conservative state
    (``gamma``: the ideal-gas ratio or an EOS object): V = m/rho, P from
    E - rho|V|^2/2 through the EOS, a^2 = (dP/drho)_S (Sec. 3.2; Sec. 4.2 step 2)."""
    eos = as_eos(gamma)
    nd = U.shape[0] - 2
    rho = U[0]
    V = [U[1 + d] / rho for d in range(nd)]
    v2 = sum(v * v for v in V)
    P = eos.pressure(rho, U[-1] - 0.5 * rho * v2)
    a2 = eos.sound2(rho, P)
    return rho, V, v2, P, a2


def _speed(v2: torch.Tensor) -> torch.Tensor:
    """|V| of c_tot = |V| + a/xi (Sec. 4.2, reading 2), with a zero
    (sub)gradient at V = 0 (adjoint reading)."""
    pos = v2 > 0
    return torch.sqrt(torch.where(pos, v2, torch.ones_like(v2))) * pos


def xi_of(a2: torch.Tensor, xi, cmax=None):
    """Reduction rate: the constant xi, or xi = [1 + (a/C_max)^4]^(1/4) (Eq. cx, Sec. 4.3)."""
    if cmax is None:
        return xi
    return (1.0 + (a2 / (cmax * cmax)) ** 2) ** 0.25


def c_tot(U: torch.Tensor, gamma: float, xi, cmax=None) -> torch.Tensor:
    """Approximate RSST characteristic speed |V| + a/xi (Sec. 4.2)."""
    rho, V, v2, P, a2 = primitives(U, gamma)
    return _speed(v2) + torch.sqrt(a2) / xi_of(a2, xi, cmax)


def physical_flux(U: torch.Tensor, d: int, gamma: float) -> torch.Tensor:
    """Euler flux along dimension d: (m_d, m V_d + P e_d, (E + P) V_d) (Eq. pvs_dt0)."""
    rho, V, v2, P, a2 = primitives(U, gamma)
    nd = U.shape[0] - 2
    vd = V[d]
    comps = [U[1 + d]]
    for e in range(nd):
        fe = U[1 + e] * vd
        if e == d:
            fe = fe + P
        comps.append(fe)
    comps.append((U[-1] + P) * vd)
    return torch.stack(comps)


# ---------------------------------------------------------------------------
# Spatial discretisation (Sec. 4.2, steps 2-5)
# ---------------------------------------------------------------------------

def mc_limiter(a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """Monotonized-central slope, named in Sec. 4.2 (reading 1): 0 if ab <= 0,
    else the smallest in magnitude of 2a, 2b, (a+b)/2 (ties resolved in that
    order)."""
    aa = 2.0 * a.abs()
    bb = 2.0 * b.abs()
    cc = 0.5 * (a + b).abs()
    pick_a = (aa <= bb) & (aa <= cc)
    pick_b = (~pick_a) & (bb <= cc)
    s = torch.where(pick_a, 2.0 * a, torch.where(pick_b, 2.0 * b, 0.5 * (a + b)))
    return torch.where(a * b > 0, s, torch.zeros_like(s))


def llf_flux(UL: torch.Tensor, UR: torch.Tensor, d: int, gamma: float, xi, cmax=None) -> torch.Tensor:
    """Local Lax-Friedrichs flux with alpha = max(c_tot(U_L), c_tot(U_R)) (Sec. 4.2, step 4);
    under the C_max law xi is evaluated on each side's own state."""
    cl = c_tot(UL, gamma, xi, cmax)
    cr = c_tot(UR, gamma, xi, cmax)
    alpha = torch.where(cl >= cr, cl, cr)
    return 0.5 * (physical_flux(UL, d, gamma) + physical_flux(UR, d, gamma)) - 0.5 * alpha * (UR - UL)


def _background_state(prob: Problem, k_lo: int, count: int) -> Optional[torch.Tensor]:
    """Background U0 = (rho0, 0, P0/(gamma-1)) at padded vertical indices
    k_lo..k_lo+count-1 (padded index = interior index + 2); it enters the
    wall ghosts of reading 7 (hydrostatic walls, App. B setting)."""
    if prob.bg_rho is None:
        return None
    rho0 = prob.bg_rho[k_lo:k_lo + count].to(DT)
    e0 = as_eos(prob.gamma).internal_energy(rho0, prob.bg_p[k_lo:k_lo + count].to(DT))
    comps = [rho0] + [torch.zeros_like(rho0)] * prob.ndim + [e0]
    return torch.stack(comps)  # [nvar, count]


def _expand_profile(vec: torch.Tensor, prob: Problem, like_ax: int, shape) -> torch.Tensor:
    """Broadcast a [nvar, count] profile along tensor axis like_ax to ``shape``."""
    view = [vec.shape[0]] + [1] * (len(shape) - 1)
    view[like_ax] = vec.shape[1]
    return vec.reshape(view).expand(shape)


def pad_axis(U: torch.Tensor, d: int, prob: Problem) -> torch.Tensor:
    """Add two ghost cells at each end of dimension d (boundary readings in the module docstring)."""
    ax = prob.axis(d)
    n = U.shape[ax]
    if prob.bc[d] == PERIODIC:
        return torch.cat([U.narrow(ax, n - 2, 2), U, U.narrow(ax, 0, 2)], dim=ax)
    # reflecting wall: ghost -1-i mirrors i (lo), ghost n+i mirrors n-1-i (hi)
    lo = torch.flip(U.narrow(ax, 0, 2), dims=[ax])
    hi = torch.flip(U.narrow(ax, n - 2, 2), dims=[ax])
    sign = torch.ones(U.shape[0], dtype=U.dtype)
    sign[1 + d] = -1.0
    sview = [U.shape[0]] + [1] * (U.dim() - 1)
    lo = lo * sign.reshape(sview)
    hi = hi * sign.reshape(sview)
    if prob.bg_rho is not None and d == prob.vertical:
        # ghost = U0(ghost) + mirror(U - U0)(image); mirror(U0) = U0 since m0 = 0
        g_lo = _background_state(prob, 0, 2)            # padded 0,1 = ghosts -2,-1
        i_lo = torch.flip(_background_state(prob, 2, 2), dims=[1])   # images 1,0
        g_hi = _background_state(prob, n + 2, 2)        # ghosts n, n+1
        i_hi = torch.flip(_background_state(prob, n, 2), dims=[1])   # images n-1, n-2
        lo = lo + _expand_profile(g_lo - i_lo, prob, ax, lo.shape)
        hi = hi + _expand_profile(g_hi - i_hi, prob, ax, hi.shape)
    return torch.cat([lo, U, hi], dim=ax)


def face_fluxes(U: torch.Tensor, d: int, prob: Problem) -> torch.Tensor:
    """LLF fluxes at the n+1 faces -1/2 .. n-1/2 of dimension d (Sec. 4.2, steps 2-4)."""
    ax = prob.axis(d)
    Up = pad_axis(U, d, prob)
    n = U.shape[ax]
    left = Up.narrow(ax, 0, n + 2)
    mid = Up.narrow(ax, 1, n + 2)
    right = Up.narrow(ax, 2, n + 2)
    sigma = mc_limiter(mid - left, right - mid)          # cells -1 .. n
    UL = (mid + 0.5 * sigma).narrow(ax, 0, n + 1)        # face i+1/2 uses cell i
    UR = (mid - 0.5 * sigma).narrow(ax, 1, n + 1)        # and cell i+1
    return llf_flux(UL, UR, d, prob.gamma, prob.xi, prob.cmax)


def euler_tendency(U: torch.Tensor, prob: Problem) -> torch.Tensor:
    """dU = -sum_d (F_{i+1/2} - F_{i-1/2}) / dx_d (Eq. pvs_dt0; Sec. 4.2 step 5)."""
    dU = torch.zeros_like(U)
    for d in range(prob.ndim):
        ax = prob.axis(d)
        F = face_fluxes(U, d, prob)
        n = U.shape[ax]
        dU = dU - (F.narrow(ax, 1, n) - F.narrow(ax, 0, n)) / prob.dx[d]
    return dU


# ---------------------------------------------------------------------------
# RSST correction (Sec. 3.2 Eqs. pvs_dt / pvs_dt_dpr / pvs_cons_rhs; App. A)
# ---------------------------------------------------------------------------

def pressure_tendency(U: torch.Tensor, dU: torch.Tensor, gamma) -> torch.Tensor:
    """dP = [(de/dP)_rho]^-1 {[V^2/2 - (de/drho)_P] drho - V.dm + dE} (Eq. pvs_dt_dpr)."""
    eos = as_eos(gamma)
    rho, V, v2, P, a2 = primitives(U, eos)
    nd = U.shape[0] - 2
    vdm = sum(V[e] * dU[1 + e] for e in range(nd))
    return ((0.5 * v2 - eos.de_drho(rho, P)) * dU[0] - vdm + dU[-1]) / eos.de_dP(rho, P)


def correction_vector(U: torch.Tensor, variant: int, gamma: float):
    """(s-selector, r): the tendency is dU - f * s * r with s = dP ('P') or drho ('rho').

    PVS: r = (1/a^2, V/a^2, (e+P+rho V^2/2)/(rho a^2))   Eq. pvs_cons_rhs
    DVS: r = (1, V, (e+P+rho V^2/2)/rho)                 App. A.1
    PMS: r = (1/a^2, 0, (e+P-rho V^2/2)/(rho a^2))       App. A.2
    DMS: r = (1, 0, (e+P-rho V^2/2)/rho)                 App. A.3
    PD : r = (0, 0, (de/dP)_rho = 1/(gamma-1))           App. A.4
    """
    eos = as_eos(gamma)
    rho, V, v2, P, a2 = primitives(U, eos)
    nd = U.shape[0] - 2
    e = eos.internal_energy(rho, P)
    one = torch.ones_like(rho)
    zero = torch.zeros_like(rho)
    if variant == PVS:
        return "P", [one / a2] + [V[k] / a2 for k in range(nd)] + [(e + P + 0.5 * rho * v2) / (rho * a2)]
    if variant == DVS:
        return "rho", [one] + [V[k] for k in range(nd)] + [(e + P + 0.5 * rho * v2) / rho]
    if variant == PMS:
        return "P", [one / a2] + [zero] * nd + [(e + P - 0.5 * rho * v2) / (rho * a2)]
    if variant == DMS:
        return "rho", [one] + [zero] * nd + [(e + P - 0.5 * rho * v2) / rho]
    if variant == PD:
        return "P", [zero] * (nd + 1) + [eos.de_dP(rho, P) * one]
    raise ValueError(f"no correction vector for variant {variant}")


def rsst_correct(U: torch.Tensor, dU: torch.Tensor, variant: int, gamma: float, xi, cmax=None) -> torch.Tensor:
    """Reduced tendency dU - (1 - 1/xi^2) s r (Sec. 4.2 steps 6-7; Eq. pvs_dt and App. A);
    under the C_max law xi is that of the cell's own sound speed."""
    if variant == EULER:
        return dU
    if cmax is None:
        f = 1.0 - 1.0 / (xi * xi)
    else:
        a2 = primitives(U, gamma)[4]
        xc = xi_of(a2, xi, cmax)
        f = 1.0 - 1.0 / (xc * xc)
    which, r = correction_vector(U, variant, gamma)
    s = pressure_tendency(U, dU, gamma) if which == "P" else dU[0]
    return torch.stack([dU[k] - f * s * r[k] for k in range(U.shape[0])])


def gravity_source(U: torch.Tensor, prob: Problem) -> torch.Tensor:
    """(0, rho F, m.F) of App. B (the force is a constant acceleration F = grav)."""
    nd = prob.ndim
    g = [float(prob.grav[d]) for d in range(nd)]
    comps = [torch.zeros_like(U[0])]
    for d in range(nd):
        comps.append(U[0] * g[d])
    comps.append(sum(U[1 + d] * g[d] for d in range(nd)))
    return torch.stack(comps)


def has_gravity(prob: Problem) -> bool:
    return any(float(prob.grav[d]) != 0.0 for d in range(prob.ndim))


def rhs(U: torch.Tensor, prob: Problem) -> torch.Tensor:
    """L(U) of Sec. 4.2 steps 2-7: Euler tendency (Eq. pvs_dt0), the RSST
    correction of the chosen form (Sec. 3.2, App. A), then the external
    force (App. B)."""
    out = rsst_correct(U, euler_tendency(U, prob), prob.variant, prob.gamma, prob.xi, prob.cmax)
    if has_gravity(prob):
        out = out + gravity_source(U, prob)
    return out


# ---------------------------------------------------------------------------
# Time integration (Sec. 4.2 steps 1 and 8)
# ---------------------------------------------------------------------------

def cfl_dt(U: torch.Tensor, prob: Problem) -> float:
    """dt = C / max_cells sum_d c_tot / dx_d with C = prob.cfl (Courant
    number 0.4 of Sec. 4.2; the multi-dimensional sum is reading 3), or with
    prob.cfl_rule = 1 the other reading, dt = C min_d dx_d / max_cells c_tot."""
    with torch.no_grad():
        c = c_tot(U, prob.gamma, float(prob.xi), prob.cmax)
        if prob.cfl_rule == 1:
            return float(prob.cfl * min(float(prob.dx[d]) for d in range(prob.ndim)) / c.max())
        rate = sum(c / prob.dx[d] for d in range(prob.ndim))
        return float(prob.cfl / rate.max())


def ssp_rk2_step(U: torch.Tensor, dt, prob: Problem) -> torch.Tensor:
    """Second-order SSP Runge-Kutta, Shu-Osher form (Sec. 4.2 step 8, which
    cites Gottlieb et al. without printing it; reading 4)."""
    Us = U + dt * rhs(U, prob)
    return 0.5 * U + 0.5 * (Us + dt * rhs(Us, prob))


def run(U: torch.Tensor, prob: Problem, nsteps: int, dt: Optional[float] = None,
        check: bool = True) -> torch.Tensor:
    """nsteps SSP-RK2 steps (Sec. 4.2); dt from the CFL rule each step when
    dt is None."""
    for _ in range(nsteps):
        h = cfl_dt(U, prob) if dt is None else dt
        U = ssp_rk2_step(U, h, prob)
        if check:
            check_physical(U, prob)
    return U


def check_physical(U: torch.Tensor, prob: Problem) -> None:
    """Raise if any cell has rho <= 0, P <= 0 or a non-finite value (no floors are applied)."""
    with torch.no_grad():
        rho, V, v2, P, a2 = primitives(U, prob.gamma)
        bad = (~torch.isfinite(U).all(dim=0)) | (rho <= 0) | (P <= 0)
        if bool(bad.any()):
            raise FloatingPointError("non-physical state (rho <= 0, P <= 0 or NaN)")


# ---------------------------------------------------------------------------
# Diagnostics
# ---------------------------------------------------------------------------

def conserved_sums(U: torch.Tensor, prob: Problem):
    """Exactly rounded sum of each conserved variable times the cell volume (math.fsum)."""
    vol = prob.cell_volume()
    return [math.fsum(U[k].reshape(-1).tolist()) * vol for k in range(U.shape[0])]


def kinetic_energy(U: torch.Tensor, prob: Problem) -> torch.Tensor:
    """J = sum_cells |m|^2 / (2 rho) * cell volume."""
    m2 = sum(U[1 + d] * U[1 + d] for d in range(prob.ndim))
    return (0.5 * m2 / U[0]).sum() * prob.cell_volume()


def kinetic_energy_gradient(U: torch.Tensor, prob: Problem) -> torch.Tensor:
    """dJ/dU of kinetic_energy: (-|V|^2/2, V, 0) * cell volume."""
    rho, V, v2, P, a2 = primitives(U, prob.gamma)
    vol = prob.cell_volume()
    return torch.stack([-0.5 * v2 * vol] + [V[d] * vol for d in range(prob.ndim)]
                       + [torch.zeros_like(rho)])
