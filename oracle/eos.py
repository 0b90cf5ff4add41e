"""Equations of state beyond the ideal gas for the oracle (TEST
INFRASTRUCTURE ONLY; the product never imports this package).

The paper states the reduced equations and the pressure tendency for any EOS
(Sec. 3.2, Eqs. pvs_cons_dpr and pvs_cons_therm) and names no non-ideal gas
with parameters, so the gas used to exercise the general formulas is this
repository's choice: the covolume (Noble-Abel) gas, P (1/rho - b) = (gamma-1)
e/rho per unit mass, i.e. with e the internal energy per volume
  P = (gamma - 1) e / (1 - b rho),
  a^2 = (dP/drho)_S = gamma P / (rho (1 - b rho)),
  (de/dP)_rho = (1 - b rho)/(gamma - 1),  (de/drho)_P = -b P/(gamma - 1).
b = 0 is the ideal gas."""


class NobleAbel:
    """Covolume gas with the oracle's EOS interface (see rsst_oracle.IdealGas)."""

    def __init__(self, gamma: float, b: float):
        self.gamma, self.b = float(gamma), float(b)

    def pressure(self, rho, eint):
        return (self.gamma - 1.0) * eint / (1.0 - self.b * rho)

    def internal_energy(self, rho, P):
        return P * (1.0 - self.b * rho) / (self.gamma - 1.0)

    def sound2(self, rho, P):
        return self.gamma * P / (rho * (1.0 - self.b * rho))

    def de_dP(self, rho, P):
        return (1.0 - self.b * rho) / (self.gamma - 1.0)

    def de_drho(self, rho, P):
        return -self.b * P / (self.gamma - 1.0)
