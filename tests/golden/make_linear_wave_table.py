"""Writes tests/golden/linear_wave_oracle_l1.json: the oracle's L1 errors of
the linear entropy-wave study (Sec. 4.4's convergence test, the workload of
paper_1812_04135_gb300.inputs.linear_wave_2d: 30 degrees, xi = 5,
P = 1000, unit time, fixed dt = 1/ceil(1/dt_CFL)) for DVS, DMS and PVS at
N = 64, 128, 256 and two amplitudes, eps = 1e-5 and 1e-6.  It calls only the
oracle (test infrastructure); about an hour on 8 cores.

  python tests/golden/make_linear_wave_table.py
"""
import json
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import torch  # noqa: E402

from oracle import rsst_oracle as ro  # noqa: E402
from oracle.workload import problem_from  # noqa: E402
from paper_1812_04135_gb300 import inputs  # noqa: E402

FORMS = ("dvs", "dms", "pvs")
NS = (64, 128, 256)
EPS = (1e-5, 1e-6)


def fields(U, gamma, th):
    """S = ln P - gamma ln rho, V_perp, rho, P of a 2D state."""
    rho = U[0]
    vx, vy = U[1] / rho, U[2] / rho
    P = (gamma - 1.0) * (U[3] - 0.5 * rho * (vx * vx + vy * vy))
    return {"S": torch.log(P) - gamma * torch.log(rho), "Vperp": -vx * math.sin(th) + vy * math.cos(th),
            "rho": rho, "P": P}


def l1_errors(var, n, eps):
    w = inputs.linear_wave_2d(n, var, eps=eps)
    prob, U0 = problem_from(w)
    nsteps = math.ceil(1.0 / ro.cfl_dt(U0, prob))
    U1 = ro.run(U0, prob, nsteps, dt=1.0 / nsteps)
    th = math.radians(30.0)
    f0, f1 = fields(U0, w["gamma"], th), fields(U1, w["gamma"], th)
    return {k: float((f1[k] - f0[k]).abs().mean()) for k in f0}


def main():
    out = {"description": "oracle L1 errors (volume average of |final - initial|) after unit time, "
                          "linear_wave_2d(n, form, eps=eps), written by tests/golden/make_linear_wave_table.py",
           "errors": {}}
    for var in FORMS:
        for eps in EPS:
            for n in NS:
                out["errors"][f"{var}:{eps:g}:{n}"] = l1_errors(var, n, eps)
                print(var, eps, n, out["errors"][f"{var}:{eps:g}:{n}"], flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "linear_wave_oracle_l1.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
