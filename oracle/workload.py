"""Turn a workload dict from ``paper_1812_04135_gb300.inputs`` into an oracle
``Problem`` plus a float64 CPU tensor (TEST INFRASTRUCTURE ONLY)."""
from __future__ import annotations

from dataclasses import replace

import torch

from . import rsst_oracle as ro
from .eos import NobleAbel

VARIANTS = {"euler": ro.EULER, "dvs": ro.DVS, "pvs": ro.PVS, "dms": ro.DMS, "pms": ro.PMS, "pd": ro.PD}
BCS = {"periodic": ro.PERIODIC, "reflect": ro.REFLECT}


def problem_from(w: dict, **over):
    v = w["variant"]
    prob = ro.Problem(
        ndim=w["ndim"], n=tuple(w["n"]), dx=tuple(w["dx"]),
        gamma=NobleAbel(w["gamma"], w["covolume"]) if w.get("covolume") else w["gamma"], xi=w["xi"],
        variant=VARIANTS[v] if isinstance(v, str) else int(v),
        grav=tuple(w["grav"]), bc=tuple(BCS[b] for b in w["bc"]), cfl=w.get("cfl", 0.4),
        vertical=w["vertical"],
        bg_rho=None if w["bg_rho"] is None else torch.as_tensor(w["bg_rho"], dtype=ro.DT),
        bg_p=None if w["bg_p"] is None else torch.as_tensor(w["bg_p"], dtype=ro.DT),
        cmax=w.get("cmax") or None,
        cfl_rule=int(w.get("cfl_rule", 0)),
    )
    if over:
        if "variant" in over and isinstance(over["variant"], str):
            over["variant"] = VARIANTS[over["variant"]]
        prob = replace(prob, **over)
    U = torch.as_tensor(w["U"], dtype=ro.DT).clone()
    return prob, U
