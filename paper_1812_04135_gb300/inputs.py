"""Seeded synthetic initial states for the RSST step.

This module only builds initial data (numpy float64, host memory) and the
run parameters that go with it.  It holds none of the method's arithmetic
(no flux, limiter, correction or time step), so both the CUDA path and the
CPU oracle can take their inputs from it.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15,
then the 64-bit finaliser with shifts 30/27/31; a double in [0, 1) is the top
53 bits times 2^-53.

Every workload returns a dict with:
  ndim, n (x, y, z order), dx, gamma, xi, variant (name), bc (per axis:
  'periodic' | 'reflect'), grav (3 entries), vertical (axis or -1),
  bg_rho / bg_p (background profiles with 2 ghost cells per end, or None),
  U (float64 array [nvar, (nz,) (ny,) nx]; components rho, m_x.., E).
"""
from __future__ import annotations

import math
from typing import Dict, List

import numpy as np

_M64 = (1 << 64) - 1


def splitmix64(seed: int, count: int) -> np.ndarray:
    """``count`` successive SplitMix64 outputs for the given seed (uint64)."""
    state = np.uint64(seed & _M64)
    idx = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = state + idx * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int) -> np.ndarray:
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_pm1(seed: int, count: int) -> np.ndarray:
    """iid U[-1, 1) doubles."""
    return 2.0 * uniform01(seed, count) - 1.0


def _centres(n: int, length: float, origin: float = 0.0) -> np.ndarray:
    return origin + (np.arange(n, dtype=np.float64) + 0.5) * (length / n)


def _pack(rho, vel, p, gamma) -> np.ndarray:
    """Conservative state from primitives: (rho, rho V, P/(gamma-1) + rho |V|^2 / 2)."""
    v2 = sum(v * v for v in vel)
    comps = [rho] + [rho * v for v in vel] + [p / (gamma - 1.0) + 0.5 * rho * v2]
    return np.ascontiguousarray(np.stack(comps).astype(np.float64))


def _base(ndim, n, dx, gamma, xi, variant, bc, grav=(0.0, 0.0, 0.0), vertical=-1,
          bg_rho=None, bg_p=None, U=None, name=""):
    return dict(name=name, ndim=ndim, n=tuple(int(v) for v in n), dx=tuple(float(h) for h in dx),
                gamma=float(gamma), xi=float(xi), variant=variant, bc=tuple(bc),
                grav=tuple(float(g) for g in grav) + (0.0,) * (3 - len(grav)),
                vertical=int(vertical), bg_rho=bg_rho, bg_p=bg_p, U=U)


# ---------------------------------------------------------------------------
# 1D periodic ideal gas: sound eigenmode and advected entropy (contact) jump
# ---------------------------------------------------------------------------

def sound_wave_1d(n: int = 256, xi: float = 1.0, variant: str = "pvs", eps: float = 1e-6,
                  gamma: float = 5.0 / 3.0) -> Dict:
    """Uniform gas at rest (rho = 1, P = 1/gamma so a = 1) plus the right-going
    linear sound eigenmode of the reduced system, wavelength = domain [0, 1):
    drho = eps rho sin(2 pi x), dV = xi a eps sin(2 pi x), dP = a^2 drho."""
    x = _centres(n, 1.0)
    w = np.sin(2.0 * math.pi * x)
    rho0, p0 = 1.0, 1.0 / gamma
    a = math.sqrt(gamma * p0 / rho0)
    rho = rho0 * (1.0 + eps * w)
    vel = xi * a * eps * w
    p = p0 * (1.0 + gamma * eps * w)
    return _base(1, (n,), (1.0 / n,), gamma, xi, variant, ("periodic",),
                 U=_pack(rho, [vel], p, gamma), name="sound_wave_1d")


def contact_1d(n: int = 256, xi: float = 1.0, variant: str = "pvs", ratio: float = 10.0,
               u: float = 0.01, gamma: float = 5.0 / 3.0) -> Dict:
    """Density rho = ratio on [0.25, 0.75) and 1 elsewhere, uniform P = 1/gamma
    (sound speed 1 in the light gas) and uniform velocity u."""
    x = _centres(n, 1.0)
    rho = np.where((x >= 0.25) & (x < 0.75), ratio, 1.0)
    p = np.full(n, 1.0 / gamma)
    vel = np.full(n, u)
    return _base(1, (n,), (1.0 / n,), gamma, xi, variant, ("periodic",),
                 U=_pack(rho, [vel], p, gamma), name="contact_1d")


def sod_1d(n: int = 256, gamma: float = 1.4) -> Dict:
    """Sod shock tube on [0, 1], diaphragm at 0.5, reflecting ends, xi = 1."""
    x = _centres(n, 1.0)
    left = x < 0.5
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    return _base(1, (n,), (1.0 / n,), gamma, 1.0, "euler", ("reflect",),
                 U=_pack(rho, [np.zeros(n)], p, gamma), name="sod_1d")


# ---------------------------------------------------------------------------
# 2D periodic shear layer (tanh interfaces, low Mach)
# ---------------------------------------------------------------------------

def shear_profile(y: np.ndarray, ratio: float, width: float = 0.02) -> np.ndarray:
    """1 outside and ``ratio`` inside the band 0.25 < y < 0.75, tanh edges."""
    band = np.tanh((y - 0.25) / width) - np.tanh((y - 0.75) / width)
    return 1.0 + 0.5 * (ratio - 1.0) * band


def shear_layer_2d(nx: int = 512, ny: int = 512, xi: float = 30.0, variant: str = "pvs",
                   ratio: float = 10.0, mach: float = 0.01, width: float = 0.02,
                   seed: int = 2, gamma: float = 5.0 / 3.0) -> Dict:
    """Periodic [0,1)^2; rho from ``shear_profile``; P = 1; V_x = +U in the
    dense band, -U outside (tanh edges), U = mach * c_dense; V_x and V_y get
    iid U[-1,1) perturbations of 1e-4 c_dense (SplitMix64 ``seed``).
    The at-rest y profile (rho(y), P = 1) is returned as the background."""
    y = _centres(ny, 1.0)
    prof = shear_profile(y, ratio, width)
    c_dense = math.sqrt(gamma * 1.0 / ratio) if ratio > 0 else 1.0
    U0 = mach * c_dense
    band = np.tanh((y - 0.25) / width) - np.tanh((y - 0.75) / width)
    vx_row = U0 * (band - 1.0)
    noise = uniform_pm1(seed, 2 * nx * ny).reshape(2, ny, nx) * (1e-4 * c_dense)
    rho = np.repeat(prof[:, None], nx, axis=1)
    vx = vx_row[:, None] + noise[0]
    vy = noise[1]
    p = np.ones((ny, nx))
    yg = _centres(ny + 4, (ny + 4) / ny, origin=-2.0 / ny)
    return _base(2, (nx, ny), (1.0 / nx, 1.0 / ny), gamma, xi, variant, ("periodic", "periodic"),
                 vertical=1, bg_rho=shear_profile(yg, ratio, width), bg_p=np.ones(ny + 4),
                 U=_pack(rho, [vx, vy], p, gamma), name="shear_layer_2d")


# ---------------------------------------------------------------------------
# Polytropic stratification under gravity (3D box and 2D adjoint case)
# ---------------------------------------------------------------------------

def polytrope_profile(z: np.ndarray, contrast: float, index: float = 1.5, g: float = 1.0):
    """Hydrostatic polytrope with top at z = 1: theta = P/rho = theta_t + g (1 - z)/(n+1),
    rho = (theta/theta_t)^n, so rho(0)/rho(1) = contrast; returns (rho, P)."""
    theta_t = g / (index + 1.0) / (contrast ** (1.0 / index) - 1.0)
    theta = theta_t + g * (1.0 - z) / (index + 1.0)
    if np.any(theta <= 0.0):
        raise ValueError("polytrope temperature <= 0 at a ghost cell: grid too coarse for this contrast")
    rho = (theta / theta_t) ** index
    return rho, rho * theta


def polytrope_3d(nx: int = 256, ny: int = 128, nz: int = 128, xi: float = 50.0,
                 variant: str = "pvs", contrast: float = 100.0, amp: float = 1e-3,
                 seed: int = 3, gamma: float = 5.0 / 3.0) -> Dict:
    """Box [0, 2] x [0, 1] x [0, 1] (dx = 1/nz), gravity -z, periodic x/y,
    reflecting z walls; entropy perturbation drho/rho = amp U[-1,1) at fixed P, V = 0."""
    h = 1.0 / nz
    z = _centres(nz, 1.0)
    rho_z, p_z = polytrope_profile(z, contrast)
    noise = uniform_pm1(seed, nx * ny * nz).reshape(nz, ny, nx)
    rho = rho_z[:, None, None] * (1.0 + amp * noise)
    p = np.broadcast_to(p_z[:, None, None], rho.shape)
    zero = np.zeros_like(rho)
    zg = _centres(nz + 4, (nz + 4) * h, origin=-2.0 * h)
    bg_rho, bg_p = polytrope_profile(zg, contrast)
    return _base(3, (nx, ny, nz), (h, h, h), gamma, xi, variant,
                 ("periodic", "periodic", "reflect"), grav=(0.0, 0.0, -1.0), vertical=2,
                 bg_rho=bg_rho, bg_p=bg_p, U=_pack(rho, [zero, zero, zero], p, gamma),
                 name="polytrope_3d")


def polytrope_2d(nx: int = 256, ny: int = 256, xi: float = 20.0, variant: str = "pvs",
                 contrast: float = 20.0, amp: float = 1e-3, seed: int = 5,
                 gamma: float = 5.0 / 3.0) -> Dict:
    """[0,1]^2, gravity -y, periodic x, reflecting y walls; entropy perturbation
    drho/rho = amp U[-1,1) at fixed P, V = 0 (the adjoint workload)."""
    h = 1.0 / ny
    y = _centres(ny, 1.0)
    rho_y, p_y = polytrope_profile(y, contrast)
    noise = uniform_pm1(seed, nx * ny).reshape(ny, nx)
    rho = rho_y[:, None] * (1.0 + amp * noise)
    p = np.broadcast_to(p_y[:, None], rho.shape)
    zero = np.zeros_like(rho)
    yg = _centres(ny + 4, (ny + 4) * h, origin=-2.0 * h)
    bg_rho, bg_p = polytrope_profile(yg, contrast)
    return _base(2, (nx, ny), (1.0 / nx, h), gamma, xi, variant, ("periodic", "reflect"),
                 grav=(0.0, -1.0, 0.0), vertical=1, bg_rho=bg_rho, bg_p=bg_p,
                 U=_pack(rho, [zero, zero], p, gamma), name="polytrope_2d")


# ---------------------------------------------------------------------------
# Batched: many independent shear layers of uneven size, xi and density ratio
# ---------------------------------------------------------------------------

BATCH_SIZES = (128, 192, 256, 384, 512, 768, 1024)
BATCH_XI = (1.0, 3.0, 10.0, 30.0)
BATCH_RATIO = (1.0, 3.0, 10.0, 100.0)


def batched_runs(count: int = 64, seed: int = 4, sizes=BATCH_SIZES, variant: str = "pvs",
                 max_size: int = 0) -> List[Dict]:
    """``count`` shear layers; size N (N x N grid), xi and density ratio drawn
    with SplitMix64 ``seed`` from BATCH_SIZES, BATCH_XI, BATCH_RATIO.
    ``max_size`` > 0 clips N (small parity cases)."""
    draws = splitmix64(seed, 3 * count).reshape(count, 3)
    runs = []
    for i in range(count):
        n = sizes[int(draws[i, 0] % np.uint64(len(sizes)))]
        if max_size:
            n = min(n, max_size)
        xi = BATCH_XI[int(draws[i, 1] % np.uint64(len(BATCH_XI)))]
        ratio = BATCH_RATIO[int(draws[i, 2] % np.uint64(len(BATCH_RATIO)))]
        w = shear_layer_2d(n, n, xi=xi, variant=variant, ratio=ratio, seed=1000 + i)
        w["name"] = f"batch[{i}]"
        runs.append(w)
    return runs


def uniform_state(ndim: int, n, xi: float = 10.0, variant: str = "pvs", rho: float = 1.3,
                  vel=(0.1, -0.05, 0.02), p: float = 0.7, gamma: float = 5.0 / 3.0) -> Dict:
    shape = tuple(reversed(tuple(n)))
    comps = [np.full(shape, rho)]
    for d in range(ndim):
        comps.append(np.full(shape, rho * vel[d]))
    v2 = sum(vel[d] ** 2 for d in range(ndim))
    comps.append(np.full(shape, p / (gamma - 1.0) + 0.5 * rho * v2))
    return _base(ndim, n, tuple(1.0 / v for v in n), gamma, xi, variant, ("periodic",) * ndim,
                 U=np.stack(comps), name="uniform")


def random_smooth_state(ndim: int, n, xi: float = 7.0, variant: str = "pvs", seed: int = 11,
                        amp: float = 0.2, gamma: float = 5.0 / 3.0, bc=None, grav=(0.0, 0.0, 0.0)) -> Dict:
    """A positive, smooth-plus-noise state for parity tests: a few random
    Fourier modes in rho, V and P plus 1e-3 iid noise."""
    shape = tuple(reversed(tuple(n)))
    coords = np.meshgrid(*[_centres(v, 1.0) for v in reversed(tuple(n))], indexing="ij")
    r = uniform_pm1(seed, 64)
    noise = uniform_pm1(seed + 1, (ndim + 2) * int(np.prod(shape))).reshape((ndim + 2,) + shape)

    def field(k, base, scale):
        ph = 0.0
        for j, c in enumerate(coords):
            ph = ph + 2.0 * math.pi * (1 + (j + k) % 2) * c + r[(7 * k + j) % 64]
        return base + scale * (amp * np.sin(ph) + 1e-3 * noise[k])

    rho = field(0, 1.0, 1.0)
    vel = [field(1 + d, 0.0, 0.5) for d in range(ndim)]
    p = field(ndim + 1, 1.0, 1.0)
    return _base(ndim, n, tuple(1.0 / v for v in n), gamma, xi, variant,
                 bc or ("periodic",) * ndim, grav=grav, U=_pack(rho, vel, p, gamma),
                 name="random_smooth")


# ---------------------------------------------------------------------------
# Linear entropy wave with velocity shear at 30 degrees (convergence study)
# ---------------------------------------------------------------------------

def linear_wave_2d(n: int, variant: str = "pvs", xi: float = 5.0, eps: float = 1e-5, p0: float = 1000.0,
                   theta_deg: float = 30.0, gamma: float = 5.0 / 3.0) -> Dict:
    """Domain [0, 1/cos t] x [0, 1/sin t], n x n cells, periodic; with
    x_par = x cos t + y sin t: rho = 1 + eps sin(2 pi x_par), P = p0,
    V_par = 1, V_perp = eps sin(2 pi x_par) (the test of the paper's linear
    wave convergence study; after unit time the exact state returns)."""
    th = math.radians(theta_deg)
    lx, ly = 1.0 / math.cos(th), 1.0 / math.sin(th)
    x = _centres(n, lx)
    y = _centres(n, ly)
    X, Y = np.meshgrid(x, y, indexing="xy")  # [ny, nx]
    xp = X * math.cos(th) + Y * math.sin(th)
    w = np.sin(2.0 * math.pi * xp)
    rho = 1.0 + eps * w
    vpar = np.ones_like(w)
    vperp = eps * w
    vx = vpar * math.cos(th) - vperp * math.sin(th)
    vy = vpar * math.sin(th) + vperp * math.cos(th)
    p = np.full_like(w, p0)
    return _base(2, (n, n), (lx / n, ly / n), gamma, xi, variant, ("periodic", "periodic"),
                 U=_pack(rho, [vx, vy], p, gamma), name="linear_wave_2d")


# ---------------------------------------------------------------------------
# Rayleigh-Taylor instability (the paper's RT test: printed initial data)
# ---------------------------------------------------------------------------

def rt_column_mass(y: np.ndarray, rho1: float = 1.0, rho2: float = 10.0, L: float = 0.025) -> np.ndarray:
    """Mass per unit area above height y (to y = 1) of the unperturbed profile,
    the closed form printed with the RT test."""
    def lncosh2(z):  # ln(e^z + e^-z), written stably
        z = np.abs(z)
        return z + np.log1p(np.exp(-2.0 * z))
    return (0.5 * (rho1 + rho2) * (1.0 - y)
            + 0.5 * L * (rho2 - rho1) * (lncosh2(0.5 / L) - lncosh2((y - 0.5) / L)))


def rayleigh_taylor_2d(n: int = 256, xi: float = 10.0, variant: str = "pvs", rho1: float = 1.0, rho2: float = 10.0,
                       L: float = 0.025, amp: float = 0.01, pc: float = 1000.0, gy: float = -1.0,
                       gamma: float = 5.0 / 3.0) -> Dict:
    """[0,1]^2, periodic x, free-slip (reflecting) y walls, gravity (0, gy):
    rho = {rho1 + (rho2 - rho1)/2 [1 + tanh((y - 1/2)/L)]} (1 + amp sin(4 pi x)),
    P = pc - m_c(y) gy (hydrostatic for the unperturbed profile), V = 0.
    The unperturbed profile is returned as the background (with wall ghosts)."""
    h = 1.0 / n
    x = _centres(n, 1.0)
    y = _centres(n, 1.0)
    prof = lambda yy: rho1 + 0.5 * (rho2 - rho1) * (1.0 + np.tanh((yy - 0.5) / L))
    eps = amp * np.sin(4.0 * math.pi * x)
    rho = prof(y)[:, None] * (1.0 + eps[None, :])
    p = np.broadcast_to((pc - rt_column_mass(y, rho1, rho2, L) * gy)[:, None], rho.shape)
    zero = np.zeros_like(rho)
    yg = _centres(n + 4, (n + 4) * h, origin=-2.0 * h)
    return _base(2, (n, n), (h, h), gamma, xi, variant, ("periodic", "reflect"), grav=(0.0, gy, 0.0), vertical=1,
                 bg_rho=prof(yg), bg_p=pc - rt_column_mass(yg, rho1, rho2, L) * gy,
                 U=_pack(rho, [zero, zero], p, gamma), name="rayleigh_taylor_2d")
