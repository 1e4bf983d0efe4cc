"""Model parameters of the 2f1s ternary phase-field model (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Phase 0 is the frozen solid, phase 1 the droplet / driving fluid (the evolved
order parameter), phase 2 the other fluid (Sec. 2.2).

* Spreading coefficients from the pairwise tensions:
  gamma_0 = s01 + s02 - s12, gamma_1 = s01 + s12 - s02, gamma_2 = s02 + s12 - s01
  (Sec. 2.1, equation below Eq. freeEnergy).
* Young's law s02 = s01 + s12 cos(theta) (Sec. 2.2) with s01 = k s12 and
  k = 9/(1+kappa) [1 + 2 sgn(theta - pi/2) sin^2(pi/4 cos theta)] (Eq. kk).
* 3/gamma_T = sum_q 1/gamma_q (Sec. 2.1, Lagrange multiplier).
* CH relation (M_cst + M_deg)/gamma_1 = (1/s_1 - 1/2) eta_1 cs2 dt (Sec. 3).
  eta_1 is called adjustable and never given a value; reading: eta_1 =
  eta_hat / gamma_1 with eta_hat = 0.1 by default.  The CH equilibrium puts
  eta mubar_1 into the second moment, which every step spreads explicitly with
  a coefficient ~ cs2 eta_hat (3D/4) / 2 on the fourth-derivative term of
  mubar_1; at D = 4, d0 = 1/2 the scheme is stable for eta_hat <= 0.1 and
  blows up within a few steps at eta_hat >= 0.3, whatever the mobility.
* Rates the paper leaves unspecified: CH s0, s2a, s2b, s3, s4 = ``s_free_ch``
  (default 1); NS s1, s3 = ``s_free_ns`` (default 1); NS s0 and s4 follow the
  local s2a (see ``lbm``).

Pinned by tests: the closed forms gamma_p(theta, k) printed in Sec. 2.2, the
identity k = 9 cos(pi/2 cos theta)/(1+kappa) for theta < 90 deg (and
9 (2 - cos(pi/2 cos theta))/(1+kappa) above), gamma_1 + gamma_2 = 2 sigma, and
Young's law recovered from the gammas.
"""
from __future__ import annotations

import dataclasses
import math


@dataclasses.dataclass
class Params:
    """Physical and numerical parameters (lattice units)."""

    W: float = 4.0                    # interface thickness D
    M_deg: float = 0.1                # degenerate mobility coefficient
    M_cst: float = 0.0                # constant mobility part
    theta_deg: float = 90.0           # contact angle of fluid 1 on the solid
    kappa: float = 0.0                # minimum dimensionless solid curvature
    sigma: float = 0.01               # fluid-fluid tension sigma_12
    rho: tuple = (1.0, 1.0, 1.0)      # densities of solid, fluid 1, fluid 2
    mu: tuple = (0.01, 0.01, 0.01)    # dynamic viscosities of solid, fluid 1, fluid 2
    d0: float = 0.5                   # scale factor, cs2 = d0
    eta_hat: float = 0.1              # eta_1 = eta_hat / gamma_1
    s_free_ch: float = 1.0            # unspecified CH rates
    s_free_ns: float = 1.0            # unspecified NS rates
    body_force: tuple = (0.0, 0.0, 0.0)
    rho_ref: float | None = None      # constant in lambda_0; None -> rho_0 (solid density)


def k_closure(theta, kappa):
    """Eq. kk: s01 / s12 as a function of contact angle and minimum curvature."""
    sgn = math.copysign(1.0, theta - math.pi / 2) if theta != math.pi / 2 else 0.0
    return 9.0 / (1.0 + kappa) * (1.0 + 2.0 * sgn * math.sin(math.pi / 4 * math.cos(theta)) ** 2)


def spreading(theta, kappa, sigma):
    """Pairwise tensions from Young's law and Eq. kk, then gamma_p (Sec. 2.1)."""
    k = k_closure(theta, kappa)
    s12 = sigma
    s01 = k * s12
    s02 = s01 + s12 * math.cos(theta)
    g0 = s01 + s02 - s12
    g1 = s01 + s12 - s02
    g2 = s02 + s12 - s01
    return k, (g0, g1, g2)


@dataclasses.dataclass
class Constants:
    k: float
    gamma: tuple
    gammaT: float
    eta: float
    s_ch: dict
    s_ns_free: dict
    cs2: float


def constants(p: Params) -> Constants:
    theta = math.radians(p.theta_deg)
    k, gam = spreading(theta, p.kappa, p.sigma)
    gT = 3.0 / sum(1.0 / g for g in gam)
    eta = p.eta_hat / gam[1]
    cs2 = p.d0
    s1 = 1.0 / (0.5 + (p.M_cst + p.M_deg) / (gam[1] * eta * cs2))
    s_ch = {"s0": p.s_free_ch, "s1": s1, "s2a": p.s_free_ch, "s2b": p.s_free_ch,
            "s3": p.s_free_ch, "s4": p.s_free_ch}
    s_ns = {"s1": p.s_free_ns, "s3": p.s_free_ns}
    return Constants(k, gam, gT, eta, s_ch, s_ns, cs2)
