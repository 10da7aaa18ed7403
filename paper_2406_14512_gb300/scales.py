"""Physical scales of an aligned pulsar magnetosphere (Sect. 2) and their
mapping to the code units of the library.

CGS formulas of Sect. 2: light-cylinder radius, Goldreich-Julian density,
plasma skin depth, polar-cap potential and Lorentz factor, pair-creation
threshold and secondary Lorentz factors, light-cylinder field and
magnetisation, current-sheet thickness, radiation-reaction-limited Lorentz
factor, spin-down power; plus the Larmor radius, plasma frequency and
synchrotron cooling time that Sect. 5.1 compares with the grid.

Code units: r* = c = e = B* = 1 (so mu = 1 and Omega = 1/R_LC in units of
r*).  The physical scale separation enters through the electron mass in
code units, m_e = Phi_pc / gamma_pc = (r*/R_LC)^2 / gamma_pc, and the
dimensionless Lorentz factors (gamma_rad, gamma_th, gamma_s) carry over
unchanged.
"""
from __future__ import annotations

import math

# CGS constants
C = 2.99792458e10          # cm / s
E = 4.80320471e-10         # statC
M_E = 9.1093837015e-28     # g
HBAR = 1.054571817e-27     # erg s
R_E = E * E / (M_E * C * C)            # classical electron radius, cm
B_QED = M_E * M_E * C ** 3 / (HBAR * E)  # critical field, G


def r_lc(period: float) -> float:
    """Light-cylinder radius c P / 2 pi (Sect. 2)."""
    return C * period / (2.0 * math.pi)


def omega(period: float) -> float:
    return 2.0 * math.pi / period


def n_gj(b: float, rlc: float) -> float:
    """Goldreich-Julian density B / (2 pi e R_LC) = Omega B / (2 pi e c)."""
    return b / (2.0 * math.pi * E * rlc)


def skin_depth(n: float, gamma: float = 1.0, mass: float = M_E) -> float:
    """Plasma skin depth sqrt(gamma m c^2 / (4 pi n e^2)) (Sect. 2)."""
    return math.sqrt(gamma * mass * C * C / (4.0 * math.pi * n * E * E))


def plasma_frequency(n: float, gamma: float = 1.0, mass: float = M_E) -> float:
    return C / skin_depth(n, gamma, mass)


def phi_pc(b_star: float, r_star: float, rlc: float) -> float:
    """Polar-cap potential drop mu Omega^2 / c^2 with Omega = c / R_LC."""
    return b_star * r_star ** 3 / (rlc * rlc)


def gamma_pc(b_star: float, r_star: float, rlc: float) -> float:
    """Lorentz factor of the full polar-cap drop e Phi_pc / m c^2."""
    return E * phi_pc(b_star, r_star, rlc) / (M_E * C * C)


def gamma_th(b_perp: float) -> float:
    """Pair-creation threshold sqrt(1 / (15 b^2)), b = B_perp / B_QED."""
    b = b_perp / B_QED
    return math.sqrt(1.0 / (15.0 * b * b))


def gamma_s(b_perp: float) -> float:
    """Lorentz factor of the secondary pairs 1 / (20 b)."""
    return 1.0 / (20.0 * b_perp / B_QED)


def b_lc(b_star: float, r_star: float, rlc: float) -> float:
    """Field at the light cylinder mu Omega^3 / c^3 = B* (r*/R_LC)^3."""
    return b_star * (r_star / rlc) ** 3


def sigma_lc(b_star: float, r_star: float, rlc: float, kappa: float, gamma_wind: float = 1.0) -> float:
    """Magnetisation at the light cylinder gamma_pc / (2 Gamma kappa)."""
    return gamma_pc(b_star, r_star, rlc) / (2.0 * gamma_wind * kappa)


def sheet_thickness(rlc: float, kappa: float, gamma_wind: float = 1.0) -> float:
    """Current-sheet thickness R_LC / (2 Gamma kappa)."""
    return rlc / (2.0 * gamma_wind * kappa)


def gamma_rad(e_par: float, b_perp: float) -> float:
    """Radiation-reaction-limited Lorentz factor sqrt(3 e E / (2 r_e^2 B^2))."""
    return math.sqrt(3.0 * E * e_par / (2.0 * R_E * R_E * b_perp * b_perp))


def spindown(b_star: float, r_star: float, rlc: float) -> float:
    """L_0 = mu^2 Omega^4 / c^3 with Omega = c / R_LC."""
    mu = b_star * r_star ** 3
    om = C / rlc
    return mu * mu * om ** 4 / C ** 3


def larmor_radius(gamma: float, b: float, mass: float = M_E) -> float:
    return gamma * mass * C * C / (E * b)


def synchrotron_time(gamma: float, b: float) -> float:
    """Cooling time 3 m c / (2 r_e^2 gamma B^2) (Sect. 5.1)."""
    return 3.0 * M_E * C / (2.0 * R_E * R_E * gamma * b * b)


def grid_steps(r_star: float, r_max: float, n: int, courant: float = 0.5):
    """Radial spacing at the star and time step of an n x n log-spherical
    grid: dr = r* (exp(ln(r_max/r*)/n) - 1), dt = courant x the 2D limit
    1 / c / sqrt(1/dr^2 + 1/(r* dtheta)^2) of the innermost cell."""
    d = math.log(r_max / r_star) / n
    dr = r_star * (math.exp(d) - 1.0)
    rdt = r_star * math.pi / n
    return dr, courant / (C * math.sqrt(1.0 / dr ** 2 + 1.0 / rdt ** 2))


def code_units(b_star: float, period: float, r_star: float = 1e6) -> dict:
    """Code-unit parameters of a pulsar: r* = c = e = B* = 1, so mu = 1 and
    Omega = r*/R_LC; the electron mass is Phi_pc / gamma_pc in these units."""
    rlc = r_lc(period)
    gpc = gamma_pc(b_star, r_star, rlc)
    phi_code = (r_star / rlc) ** 2
    return {"r_lc": rlc / r_star, "m_e": phi_code / gpc, "gamma_pc": gpc,
            "gamma_th": gamma_th(b_star), "gamma_s": gamma_s(b_star),
            "b_ref": (r_star / rlc) ** 3}
