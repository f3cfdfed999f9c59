"""Closed-form MPCD transport coefficients (test infrastructure).

Used by the oracle's pins only: the measured viscosity of a standalone MPCD
Poiseuille flow is compared with these formulas.

* SRD in 2D, kinetic plus collisional part (Kikuchi et al., the form the paper
  cites for Eq. 5; the printed Eq. 5 is garbled and is not used):
  nu_kin = (kT dt / m) [N / ((N - 1 + e^-N)(1 - cos 2 alpha)) - 1/2],
  nu_col = a^2 (1 - cos alpha)(N - 1 + e^-N) / (12 N dt).
* SRD in 3D (same source; not printed in the paper):
  nu_kin = (kT dt / 2m) [5N / ((N - 1 + e^-N)(2 - cos alpha - cos 2 alpha)) - 1],
  nu_col = a^2 (1 - cos alpha)(N - 1 + e^-N) / (18 N dt).
* MPCD-AT, Eq. 7 of the paper:
  nu = (kT dt / m) [N / (N - 1 + e^-N) - 1/2] + (a^2 / 12 dt)(N - 1 + e^-N) / N.

N is the mean number of particles per collision cell, a the cell side and dt
the MPCD time step (1 in lattice units), kT and m as in the simulation.
"""
from __future__ import annotations

import math


def srd_viscosity_2d(N: float, kT: float, alpha: float, a: float = 1.0, m: float = 1.0,
                     dt: float = 1.0) -> tuple[float, float]:
    """(kinetic, collisional) kinematic viscosity of 2D SRD."""
    s = N - 1.0 + math.exp(-N)
    kin = kT * dt / m * (N / (s * (1.0 - math.cos(2.0 * alpha))) - 0.5)
    col = a * a * (1.0 - math.cos(alpha)) * s / (12.0 * N * dt)
    return kin, col


def srd_viscosity_3d(N: float, kT: float, alpha: float, a: float = 1.0, m: float = 1.0,
                     dt: float = 1.0) -> tuple[float, float]:
    """(kinetic, collisional) kinematic viscosity of 3D SRD."""
    s = N - 1.0 + math.exp(-N)
    kin = kT * dt / (2.0 * m) * (5.0 * N / (s * (2.0 - math.cos(alpha) - math.cos(2.0 * alpha))) - 1.0)
    col = a * a * (1.0 - math.cos(alpha)) * s / (18.0 * N * dt)
    return kin, col


def at_viscosity(N: float, kT: float, a: float = 1.0, m: float = 1.0, dt: float = 1.0) -> tuple[float, float]:
    """(kinetic, collisional) kinematic viscosity of MPCD-AT, Eq. 7."""
    s = N - 1.0 + math.exp(-N)
    kin = kT * dt / m * (N / s - 0.5)
    col = a * a / (12.0 * dt) * s / N
    return kin, col


def at_kT_for_viscosity(nu: float, N: float, a: float = 1.0, m: float = 1.0, dt: float = 1.0) -> float:
    """kT that gives MPCD-AT the kinematic viscosity nu (Eq. 7 solved for kT)."""
    kin1, col = at_viscosity(N, 1.0, a, m, dt)
    return (nu - col) / kin1
