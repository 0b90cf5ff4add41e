"""Thin Python binding of librsst (C ABI in include/rsst.h).

Argument marshalling only: every step of the method runs in the CUDA
library.  Functions keep the C names (``rsst_init``, ``rsst_step``, ...);
``Solver`` wraps a handle for convenience.  If librsst.so is missing or
cannot load, every call raises: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "librsst.so")

RSST_OK, RSST_EINVAL, RSST_ECUDA, RSST_ENONPHYSICAL, RSST_ETIMEOUT, RSST_EUNSUPPORTED, RSST_ENOMEM = 0, -1, -2, -3, -4, -5, -6
ERROR_NAMES = {-1: "EINVAL", -2: "ECUDA", -3: "ENONPHYSICAL", -4: "ETIMEOUT", -5: "EUNSUPPORTED", -6: "ENOMEM"}
VARIANTS = {"euler": 0, "dvs": 1, "pvs": 2, "dms": 3, "pms": 4, "pd": 5}
PRECISIONS = {"fp64": 0, "fp32_pert": 1, "fp64_df": 2}
BCS = {"periodic": 0, "reflect": 1}


class RsstError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: RSST_{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


class Config(C.Structure):
    _fields_ = [
        ("ndim", C.c_int32), ("n", C.c_int32 * 3), ("dx", C.c_double * 3), ("bc", C.c_int32 * 3),
        ("variant", C.c_int32), ("precision", C.c_int32), ("xi", C.c_double), ("gamma", C.c_double),
        ("cfl", C.c_double), ("grav", C.c_double * 3), ("vertical", C.c_int32), ("cfl_rule", C.c_int32),
        ("bg_rho", C.POINTER(C.c_double)), ("bg_p", C.POINTER(C.c_double)), ("cmax", C.c_double),
        ("covolume", C.c_double),
    ]


_lib = None


def lib():
    """Load librsst.so once; raise if it is absent (build it with __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"librsst.so not built at {LIB_PATH}; run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, dbl = C.c_void_p, C.c_int, C.c_int64, C.c_double
        pd = C.POINTER(C.c_double)
        sig = {
            "rsst_init": (i32, [C.POINTER(vp), C.POINTER(Config), vp]),
            "rsst_destroy": (None, [vp]),
            "rsst_set_state": (i32, [vp, vp, i32]),
            "rsst_get_state": (i32, [vp, vp, i32]),
            "rsst_step": (i32, [vp, dbl, i32]),
            "rsst_set_graph_steps": (i32, [vp, i32]),
            "rsst_dt": (i32, [vp, pd]),
            "rsst_sync": (i32, [vp]),
            "rsst_debug_stall_wait": (i32, [vp, i64]),
            "rsst_batch_debug_stall_wait": (i32, [vp, i32, i64]),
            "rsst_time": (i32, [vp, pd]),
            "rsst_conserved_sums": (i32, [vp, pd]),
            "rsst_kernel_launches": (i64, [vp]),
            "rsst_conserved_sums_noalloc": (i32, [vp, i32, C.POINTER(C.c_int32), pd, vp, vp]),
            "rsst_config_size": (C.c_size_t, []),
            "rsst_math_selftest": (i32, [i32, pd, C.POINTER(C.c_int32), pd]),
            "rsst_fp64_fma_peak": (i32, [i32, pd, pd]),
            "rsst_adjoint_record": (i32, [vp, dbl, i32, i32]),
            "rsst_adjoint_segments": (i32, [vp, C.POINTER(C.c_int32)]),
            "rsst_adjoint_step": (i32, [vp, i32, vp, pd]),
            "rsst_kinetic_energy": (i32, [vp, pd, vp]),
            "rsst_adjoint_rho_fixed_vp": (i32, [vp, vp, vp, i32, C.POINTER(C.c_int32), vp]),
            "rsst_batch_init": (i32, [C.POINTER(vp), i32, C.POINTER(Config), vp]),
            "rsst_batch_destroy": (None, [vp]),
            "rsst_batch_set_state": (i32, [vp, i32, vp, i32]),
            "rsst_batch_get_state": (i32, [vp, i32, vp, i32]),
            "rsst_batch_step": (i32, [vp, i32]),
            "rsst_batch_step_looped": (i32, [vp, i32]),
            "rsst_batch_dt": (i32, [vp, pd]),
            "rsst_batch_sync": (i32, [vp]),
            "rsst_batch_autotune": (i32, [vp, i32, C.POINTER(C.c_int32), pd]),
            "rsst_batch_tile_shape": (i32, [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
            "rsst_batch_kernel_launches": (i64, [vp]),
            "rsst_last_error": (C.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        if L.rsst_config_size() != C.sizeof(Config):
            raise ImportError("rsst_config layout mismatch between librsst.so and the binding")
        _lib = L
    return _lib


def _check(rc: int, where: str) -> int:
    if rc != RSST_OK:
        raise RsstError(rc, where, lib().rsst_last_error().decode(errors="replace"))
    return rc


def make_config(ndim, n, dx, *, variant="pvs", precision="fp64", xi=1.0, gamma=5.0 / 3.0, cfl=0.4,
                grav=(0.0, 0.0, 0.0), bc=("periodic",) * 3, vertical=-1, bg_rho=None, bg_p=None, cmax=0.0,
                cfl_rule=0, covolume=0.0):
    """Build an ``rsst_config``; the returned object keeps the background arrays alive."""
    cfg = Config()
    cfg.ndim = int(ndim)
    for d in range(3):
        cfg.n[d] = int(n[d]) if d < ndim else 1
        cfg.dx[d] = float(dx[d]) if d < ndim else 1.0
        b = bc[d] if d < len(bc) else "periodic"
        cfg.bc[d] = BCS[b] if isinstance(b, str) else int(b)
        cfg.grav[d] = float(grav[d]) if d < len(grav) else 0.0
    cfg.variant = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    cfg.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    cfg.xi, cfg.gamma, cfg.cfl = float(xi), float(gamma), float(cfl)
    cfg.vertical = int(vertical)
    cfg.cmax = float(cmax or 0.0)
    cfg.cfl_rule = int(cfl_rule)
    cfg.covolume = float(covolume or 0.0)
    cfg._keep = []
    if bg_rho is not None:
        r = np.ascontiguousarray(bg_rho, dtype=np.float64)
        p = np.ascontiguousarray(bg_p, dtype=np.float64)
        if 0 <= cfg.vertical < ndim:
            need = cfg.n[cfg.vertical] + 4
            if r.shape != (need,) or p.shape != (need,):
                raise ValueError(f"background profiles need n[vertical] + 4 = {need} values "
                                 f"(got {r.shape}, {p.shape})")
        cfg._keep = [r, p]
        cfg.bg_rho = r.ctypes.data_as(C.POINTER(C.c_double))
        cfg.bg_p = p.ctypes.data_as(C.POINTER(C.c_double))
    return cfg


def config_from_workload(w: dict, precision="fp64", **over):
    args = dict(variant=w["variant"], precision=precision, xi=w["xi"], gamma=w["gamma"], cfl=w.get("cfl", 0.4),
                grav=w["grav"], bc=w["bc"], vertical=w["vertical"] if w["bg_rho"] is not None else -1,
                bg_rho=w["bg_rho"], bg_p=w["bg_p"], cmax=w.get("cmax") or 0.0, cfl_rule=w.get("cfl_rule", 0),
                covolume=w.get("covolume") or 0.0)
    args.update(over)
    return make_config(w["ndim"], w["n"], w["dx"], **args)


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


# --- the C entry points, same names -----------------------------------------

def _f64_ptr(U, where: str, on_host: bool = False) -> int:
    """Address of a contiguous float64 buffer, checked against where it must
    live: host memory (numpy array or CPU tensor) when ``on_host``, else a
    CUDA tensor.  The C ABI takes bare pointers and cannot check this."""
    if isinstance(U, np.ndarray):
        if U.dtype != np.float64 or not U.flags["C_CONTIGUOUS"]:
            raise ValueError(f"{where}: need a C-contiguous float64 array")
        if not on_host:
            raise ValueError(f"{where}: a numpy array is host memory; pass on_host=True or a CUDA tensor")
        return U.ctypes.data
    import torch
    if not isinstance(U, torch.Tensor) or U.dtype != torch.float64 or not U.is_contiguous():
        raise ValueError(f"{where}: need a contiguous float64 tensor")
    if U.is_cuda == bool(on_host):
        raise ValueError(f"{where}: tensor on {U.device} but on_host={bool(on_host)}")
    return U.data_ptr()


def rsst_init(cfg: Config, stream=None) -> int:
    h = C.c_void_p()
    _check(lib().rsst_init(C.byref(h), C.byref(cfg), _stream_ptr(stream)), "rsst_init")
    return h.value


def rsst_destroy(h: int) -> None:
    lib().rsst_destroy(h)


def rsst_set_state(h: int, U, on_host: bool = False) -> None:
    """U: float64 tensor or ndarray in the caller layout [nvar][nz][ny][nx], contiguous."""
    ptr = _f64_ptr(U, "rsst_set_state", on_host)
    _check(lib().rsst_set_state(h, ptr, int(on_host)), "rsst_set_state")


def rsst_get_state(h: int, U, on_host: bool = False) -> None:
    ptr = _f64_ptr(U, "rsst_get_state", on_host)
    _check(lib().rsst_get_state(h, ptr, int(on_host)), "rsst_get_state")


def rsst_step(h: int, dt: float = 0.0, nsteps: int = 1) -> None:
    _check(lib().rsst_step(h, float(dt), int(nsteps)), "rsst_step")


def rsst_dt(h: int) -> float:
    out = C.c_double()
    _check(lib().rsst_dt(h, C.byref(out)), "rsst_dt")
    return out.value


def rsst_time(h: int) -> float:
    t = C.c_double()
    _check(lib().rsst_time(h, C.byref(t)), "rsst_time")
    return t.value


def rsst_sync(h: int) -> None:
    _check(lib().rsst_sync(h), "rsst_sync")


def rsst_debug_stall_wait(h: int, limit_ns: int) -> None:
    """Failure-detection test hook: each tile of the 2D float32 TMA kernel
    also waits limit_ns on a barrier nothing completes (0: off)."""
    _check(lib().rsst_debug_stall_wait(h, int(limit_ns)), "rsst_debug_stall_wait")


def rsst_conserved_sums(h: int, nvar: int) -> list:
    out = (C.c_double * nvar)()
    _check(lib().rsst_conserved_sums(h, out), "rsst_conserved_sums")
    return list(out)


def rsst_conserved_sums_noalloc(U, n, dx, sums, stream=None) -> None:
    """Conservation sums without allocation: U (float64 CUDA tensor, caller
    layout) and sums (float64 CUDA tensor of nvar entries) belong to the caller."""
    ndim = len(n)
    nn = (C.c_int32 * ndim)(*[int(v) for v in n])
    dd = (C.c_double * ndim)(*[float(v) for v in dx])
    pu = _f64_ptr(U, "rsst_conserved_sums_noalloc")
    ps = _f64_ptr(sums, "rsst_conserved_sums_noalloc")
    _check(lib().rsst_conserved_sums_noalloc(pu, ndim, nn, dd, ps, _stream_ptr(stream)), "rsst_conserved_sums_noalloc")


def rsst_adjoint_record(h: int, dt: float, nsteps: int, every: int) -> None:
    _check(lib().rsst_adjoint_record(h, float(dt), int(nsteps), int(every)), "rsst_adjoint_record")


def rsst_adjoint_segments(h: int) -> int:
    n = C.c_int32()
    _check(lib().rsst_adjoint_segments(h, C.byref(n)), "rsst_adjoint_segments")
    return n.value


def rsst_adjoint_step(h: int, seg: int, lam) -> float:
    """Reverse one segment in place on ``lam`` (float64 CUDA tensor, caller layout); returns dJ/dxi of it."""
    acc = C.c_double(0.0)
    ptr = _f64_ptr(lam, "rsst_adjoint_step")
    _check(lib().rsst_adjoint_step(h, int(seg), ptr, C.byref(acc)), "rsst_adjoint_step")
    return acc.value


def rsst_adjoint_rho_fixed_vp(U, lam, out, stream=None) -> None:
    """dJ/drho at fixed V and P into ``out`` (float64 CUDA tensor of the grid's
    shape) from ``lam`` = dJ/dU and the state ``U`` (float64 CUDA tensors,
    caller layout [nvar][nz][ny][nx])."""
    ndim = U.dim() - 1
    if U.shape[0] != ndim + 2 or tuple(lam.shape) != tuple(U.shape) or tuple(out.shape) != tuple(U.shape[1:]):
        raise ValueError(f"rsst_adjoint_rho_fixed_vp: shapes {tuple(U.shape)}, {tuple(lam.shape)}, {tuple(out.shape)}")
    n = (C.c_int32 * ndim)(*[int(U.shape[ndim - d]) for d in range(ndim)])  # (x, y, z) order
    pu = _f64_ptr(U, "rsst_adjoint_rho_fixed_vp")
    pl = _f64_ptr(lam, "rsst_adjoint_rho_fixed_vp")
    po = _f64_ptr(out, "rsst_adjoint_rho_fixed_vp")
    _check(lib().rsst_adjoint_rho_fixed_vp(pu, pl, po, ndim, n, _stream_ptr(stream)), "rsst_adjoint_rho_fixed_vp")


def rsst_kinetic_energy(h: int, grad=None) -> float:
    J = C.c_double()
    ptr = None if grad is None else _f64_ptr(grad, "rsst_kinetic_energy")
    _check(lib().rsst_kinetic_energy(h, C.byref(J), ptr), "rsst_kinetic_energy")
    return J.value


def rsst_math_selftest(n: int = 1 << 20):
    ulp = C.c_double()
    bad = C.c_int32()
    rel = C.c_double()
    _check(lib().rsst_math_selftest(int(n), C.byref(ulp), C.byref(bad), C.byref(rel)), "rsst_math_selftest")
    return ulp.value, bad.value, rel.value


def rsst_fp64_fma_peak(iters: int = 20000):
    """Measured float64 FMA throughput (TFLOP/s, launch ms) of the current device."""
    tf, ms = C.c_double(), C.c_double()
    _check(lib().rsst_fp64_fma_peak(int(iters), C.byref(tf), C.byref(ms)), "rsst_fp64_fma_peak")
    return tf.value, ms.value


def rsst_set_graph_steps(h: int, k: int) -> None:
    _check(lib().rsst_set_graph_steps(h, int(k)), "rsst_set_graph_steps")


def rsst_kernel_launches(h: int) -> int:
    return int(lib().rsst_kernel_launches(h))


class Solver:
    """One run on the current CUDA device; state in and out as float64 torch tensors."""

    def __init__(self, w: dict, precision: str = "fp64", stream=None, **over):
        import torch
        lib()  # a missing library is reported as such, before the device is touched
        self.w = w
        self.ndim = w["ndim"]
        self.nvar = self.ndim + 2
        self.shape = (self.nvar,) + tuple(reversed(w["n"]))
        self.cfg = config_from_workload(w, precision=precision, **over)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.h = rsst_init(self.cfg, self.stream)

    def set_state(self, U) -> None:
        import torch
        if isinstance(U, np.ndarray):
            U = torch.from_numpy(np.ascontiguousarray(U, dtype=np.float64))
        U = U.contiguous()
        if U.dtype != torch.float64 or tuple(U.shape) != self.shape:
            raise ValueError(f"set_state: need float64 of shape {self.shape}, got {U.dtype} {tuple(U.shape)}")
        self._keep = U
        rsst_set_state(self.h, U, on_host=not U.is_cuda)

    def get_state(self, device="cuda"):
        import torch
        out = torch.empty(self.shape, dtype=torch.float64, device=device)
        rsst_get_state(self.h, out, on_host=(out.device.type == "cpu"))
        return out

    def step(self, nsteps: int = 1, dt: float = 0.0) -> None:
        rsst_step(self.h, dt, nsteps)

    def set_graph_steps(self, k: int) -> None:
        rsst_set_graph_steps(self.h, k)

    def dt(self) -> float:
        return rsst_dt(self.h)

    def sync(self) -> None:
        rsst_sync(self.h)

    def time(self) -> float:
        return rsst_time(self.h)

    def sums(self) -> list:
        return rsst_conserved_sums(self.h, self.nvar)

    def launches(self) -> int:
        return rsst_kernel_launches(self.h)

    def close(self) -> None:
        if getattr(self, "h", None):
            rsst_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --- batched runs -----------------------------------------------------------

def rsst_batch_init(cfgs, stream) -> int:
    arr = (Config * len(cfgs))(*cfgs)
    h = C.c_void_p()
    _check(lib().rsst_batch_init(C.byref(h), len(cfgs), arr, _stream_ptr(stream)), "rsst_batch_init")
    return h.value


def rsst_batch_destroy(b: int) -> None:
    lib().rsst_batch_destroy(b)


def rsst_batch_set_state(b: int, run: int, U, on_host: bool = False) -> None:
    ptr = _f64_ptr(U, "rsst_batch_set_state", on_host)
    _check(lib().rsst_batch_set_state(b, run, ptr, int(on_host)), "rsst_batch_set_state")


def rsst_batch_get_state(b: int, run: int, U, on_host: bool = False) -> None:
    ptr = _f64_ptr(U, "rsst_batch_get_state", on_host)
    _check(lib().rsst_batch_get_state(b, run, ptr, int(on_host)), "rsst_batch_get_state")


def rsst_batch_step(b: int, nsteps: int = 1) -> None:
    _check(lib().rsst_batch_step(b, int(nsteps)), "rsst_batch_step")


def rsst_batch_step_looped(b: int, nsteps: int = 1) -> None:
    _check(lib().rsst_batch_step_looped(b, int(nsteps)), "rsst_batch_step_looped")


def rsst_batch_dt(b: int, nruns: int) -> list:
    out = (C.c_double * nruns)()
    _check(lib().rsst_batch_dt(b, out), "rsst_batch_dt")
    return list(out)


def rsst_batch_sync(b: int) -> None:
    _check(lib().rsst_batch_sync(b), "rsst_batch_sync")


def rsst_batch_debug_stall_wait(b: int, run: int, limit_ns: int) -> None:
    _check(lib().rsst_batch_debug_stall_wait(b, int(run), int(limit_ns)), "rsst_batch_debug_stall_wait")


def rsst_batch_autotune(b: int, steps: int = 3):
    c = C.c_int32()
    ms = C.c_double()
    _check(lib().rsst_batch_autotune(b, int(steps), C.byref(c), C.byref(ms)), "rsst_batch_autotune")
    return c.value, ms.value


def rsst_batch_tile_shape(b: int):
    bx, by = C.c_int32(), C.c_int32()
    _check(lib().rsst_batch_tile_shape(b, C.byref(bx), C.byref(by)), "rsst_batch_tile_shape")
    return bx.value, by.value


def rsst_batch_kernel_launches(b: int) -> int:
    return int(lib().rsst_batch_kernel_launches(b))


class BatchSolver:
    """Many 2D float32-perturbation runs on one device, on a stream of their own."""

    def __init__(self, workloads, stream=None):
        import torch
        lib()  # a missing library is reported as such, before the device is touched
        self.ws = list(workloads)
        self.cfgs = [config_from_workload(w, precision="fp32_pert") for w in self.ws]
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.b = rsst_batch_init(self.cfgs, self.stream)
        self.nruns = len(self.ws)

    def set_state(self, run: int, U) -> None:
        import torch
        if isinstance(U, np.ndarray):
            U = torch.from_numpy(np.ascontiguousarray(U, dtype=np.float64))
        U = U.contiguous()
        w = self.ws[run]
        shape = (w["ndim"] + 2,) + tuple(reversed(w["n"]))
        if U.dtype != torch.float64 or tuple(U.shape) != shape:
            raise ValueError(f"set_state: need float64 of shape {shape}, got {U.dtype} {tuple(U.shape)}")
        self._keep = getattr(self, "_keep", {})
        self._keep[run] = U
        rsst_batch_set_state(self.b, run, U, on_host=not U.is_cuda)

    def get_state(self, run: int, device="cuda"):
        import torch
        w = self.ws[run]
        out = torch.empty((w["ndim"] + 2,) + tuple(reversed(w["n"])), dtype=torch.float64, device=device)
        rsst_batch_get_state(self.b, run, out, on_host=(out.device.type == "cpu"))
        return out

    def step(self, nsteps: int = 1) -> None:
        rsst_batch_step(self.b, nsteps)

    def step_looped(self, nsteps: int = 1) -> None:
        rsst_batch_step_looped(self.b, nsteps)

    def autotune(self, steps: int = 3):
        return rsst_batch_autotune(self.b, steps)

    def tile_shape(self):
        return rsst_batch_tile_shape(self.b)

    def dts(self) -> list:
        return rsst_batch_dt(self.b, self.nruns)

    def sync(self) -> None:
        rsst_batch_sync(self.b)

    def launches(self) -> int:
        return rsst_batch_kernel_launches(self.b)

    def close(self) -> None:
        if getattr(self, "b", None):
            rsst_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --- autograd ---------------------------------------------------------------

def _make_rsst_run():
    import torch

    class RsstRun(torch.autograd.Function):
        """U_N = step^N(U_0; xi) with the library's discrete adjoint as backward.

        forward(U0, xi, solver, dt, nsteps, every): the solver (a float64
        Solver whose xi equals ``xi``) records checkpoints every ``every``
        steps; backward reverses the segments (recompute + step adjoints) and
        returns dJ/dU0 and dJ/dxi.  dt is held fixed."""

        @staticmethod
        def forward(ctx, U0, xi, solver, dt, nsteps, every):
            if abs(float(xi) - solver.w["xi"]) > 0:
                raise ValueError("xi must equal the solver's xi (the kernel reads it from the handle)")
            solver.set_state(U0.detach().to(torch.float64).contiguous())
            rsst_adjoint_record(solver.h, dt, nsteps, every)
            ctx.solver = solver
            ctx.xi_device = xi.device if isinstance(xi, torch.Tensor) else None
            return solver.get_state(U0.device if U0.is_cuda else "cuda").to(U0.device)

        @staticmethod
        def backward(ctx, gN):
            s = ctx.solver
            lam = gN.detach().to(device="cuda", dtype=torch.float64).contiguous().clone()
            dxi = 0.0
            for seg in reversed(range(rsst_adjoint_segments(s.h))):
                dxi += rsst_adjoint_step(s.h, seg, lam)
            gxi = torch.tensor(dxi, dtype=torch.float64, device=ctx.xi_device) if ctx.xi_device is not None else None
            return lam.to(gN.device), gxi, None, None, None, None

    return RsstRun


_RSST_RUN = None


def rsst_run(U0, xi, solver, dt, nsteps, every):
    """Differentiable run of nsteps fixed-dt steps (see RsstRun)."""
    global _RSST_RUN
    if _RSST_RUN is None:
        _RSST_RUN = _make_rsst_run()
    return _RSST_RUN.apply(U0, xi, solver, dt, nsteps, every)
