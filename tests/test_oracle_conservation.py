"""Conservation properties by form (Sec. 5 and App. A): mass for the
density-reduced forms (constant xi), PD and xi = 1; momentum for the
momentum-conserving PMS/DMS and for PD; energy and mass in a closed
reflecting box; the pressure-reduced PVS/PMS carry a mass source."""
import math

import pytest
import torch

from oracle import rsst_oracle as ro
from oracle.workload import problem_from
from paper_1812_04135_gb300 import inputs


def _drift(w, var, nsteps=20):
    prob, U = problem_from(w, variant=var)
    s0 = ro.conserved_sums(U, prob)
    U1 = ro.run(U, prob, nsteps)
    s1 = ro.conserved_sums(U1, prob)
    scale = [math.fsum(U[k].abs().reshape(-1).tolist()) * prob.cell_volume() for k in range(U.shape[0])]
    return [(b - a) / sc for a, b, sc in zip(s0, s1, scale)]


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_conservation_by_form(ndim):
    n = {1: (64,), 2: (24, 20), 3: (10, 8, 6)}[ndim]
    w = inputs.random_smooth_state(ndim, n, xi=6.0)
    eps = 1e-13
    for var in ("euler", "dvs", "pvs", "dms", "pms", "pd"):
        d = _drift(w, var)
        mass, mom, energy = d[0], d[1:1 + ndim], d[-1]
        if var in ("euler", "dvs", "dms", "pd"):
            assert abs(mass) < eps, (var, mass)
        else:
            assert abs(mass) > 1e-8, (var, mass)       # -f dP / a^2 is a real mass source
        if var in ("euler", "pms", "dms", "pd"):
            assert max(abs(m) for m in mom) < eps, (var, mom)
        if var == "euler":
            assert abs(energy) < eps


def test_closed_reflecting_box_conserves_mass_and_energy():
    w = inputs.random_smooth_state(2, (20, 16), xi=1.0, bc=("reflect", "reflect"), variant="euler")
    d = _drift(w, "euler")
    assert abs(d[0]) < 1e-13 and abs(d[-1]) < 1e-13
    d = _drift(w, "dms")
    assert abs(d[0]) < 1e-13
