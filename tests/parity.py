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
