"""Host-side rules of arXiv 2501.05300 used to set up a simulation.

- refinement profile d(z) (Sec. 2.1, Eq. 1) and its discrete layers;
- solver iteration count N_it = 0.1 n_d / eps (Sec. 2.2, Eq. 8);
- time step dt = 1/2 sqrt(eps d / a), a = 3 sigma / (2 rho d) (Sec. 2.2, Eq. 9);
- contact-network length of a refined bed (Sec. 2.2, Eq. 10).
"""
from __future__ import annotations

import math


def refinement_profile(z: float, d_min: float, gamma: float, d_max: float) -> float:
    """Particle diameter at depth z below the surface (Eq. 1)."""
    if gamma <= 0:
        return d_min
    z_max = (d_max - d_min) / gamma
    return d_min + gamma * z if z < z_max else d_max


def z_max(d_min: float, gamma: float, d_max: float) -> float:
    """Depth at which the profile reaches d_max (Eq. 1)."""
    return (d_max - d_min) / gamma


def layer_bottoms(d0: float, growth: float, eta: float, n_layers: int) -> list[float]:
    """Depth of the bottom of layer n: z_n = sum_{i<=n} eta d_i with
    d_i = d0 growth^i (Sec. 2.1)."""
    out, z = [], 0.0
    for i in range(n_layers):
        z += eta * d0 * growth ** i
        out.append(z)
    return out


def discrete_aggressiveness(growth: float, eta: float) -> float:
    """gamma(r, eta) = (r - 1) / (r eta) of a layered bed (Sec. 2.1)."""
    return (growth - 1.0) / (growth * eta)


def n_iterations(n_d: float, eps: float = 0.02) -> int:
    """Solver iterations N_it = 0.1 n_d / eps (Eq. 8), rounded up."""
    return int(math.ceil(0.1 * n_d / eps - 1e-9))


def timestep(d: float, eps: float, rho: float, sigma: float) -> float:
    """dt = 1/2 sqrt(eps d / a) with a = 3 sigma / (2 rho d) (Eq. 9)."""
    a = 3.0 * sigma / (2.0 * rho * d)
    return 0.5 * math.sqrt(eps * d / a)


def network_length_uniform(h: float, d: float) -> float:
    """n_d = h / d for a uniform bed of height h (Sec. 2.2)."""
    return h / d


def network_length_refined(eta: float, d_min: float, d_max: float, growth: float,
                           h: float, zmax: float) -> float:
    """n_d = eta log(d_max/d_min)/log r + (h - z_max)/d_max (Eq. 10)."""
    return eta * math.log(d_max / d_min) / math.log(growth) + (h - zmax) / d_max
