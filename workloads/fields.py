"""Nodal vorticity fields for the synthetic workloads (inputs only)."""
from __future__ import annotations

import numpy as np


def uniform_field(n_nodes: int, w) -> np.ndarray:
    """The same vorticity vector ``w`` at every node."""
    return np.tile(np.asarray(w, dtype=np.float64)[None, :], (n_nodes, 1))


def constant_plus_noise(n_nodes: int, rng: np.random.Generator, base=(0.0, 0.0, 1.0), amp=0.1):
    """``base`` plus ``amp`` * N(0,1) per component."""
    return np.asarray(base, dtype=np.float64)[None, :] + amp * rng.standard_normal((n_nodes, 3))


def gaussian_ring(nodes: np.ndarray, radius=1.0, sigma=0.2, gamma=1.0, z0=0.0) -> np.ndarray:
    """Azimuthal vorticity of a Gaussian-core ring in the plane z = z0.

    omega_theta = gamma * exp(-d^2/sigma^2) / (pi sigma^2), d^2 = (rho - radius)^2 + (z - z0)^2.
    """
    x, y, z = nodes[:, 0], nodes[:, 1], nodes[:, 2]
    rho = np.hypot(x, y)
    d2 = (rho - radius) ** 2 + (z - z0) ** 2
    mag = gamma * np.exp(-d2 / sigma**2) / (np.pi * sigma**2)
    safe = np.where(rho > 0, rho, 1.0)
    et = np.stack([-y / safe, x / safe, np.zeros_like(x)], axis=1)
    et[rho == 0] = 0.0
    return mag[:, None] * et


def two_rings(nodes: np.ndarray, radius=1.0, sigma=0.15, separation=1.5) -> np.ndarray:
    """Two coaxial rings at z = -separation/2 (circulation +1) and +separation/2 (circulation -1)."""
    return gaussian_ring(nodes, radius, sigma, +1.0, -separation / 2) + gaussian_ring(
        nodes, radius, sigma, -1.0, +separation / 2
    )


def fourier_curl_field(nodes: np.ndarray, rng: np.random.Generator, n_modes=8, kmax=3):
    """Curl of a random Fourier vector potential A = sum_j a_j cos(k_j . x + phi_j).

    k_j = pi * (integer vector in [-kmax, kmax]^3 minus 0), a_j ~ N(0,1)^3 |k_j|^-2,
    phi_j ~ U[0, 2 pi).  omega = curl A = -sum_j sin(k_j . x + phi_j) k_j x a_j,
    which is divergence-free at every point.
    """
    ks = []
    while len(ks) < n_modes:
        k = rng.integers(-kmax, kmax + 1, size=3)
        if np.any(k != 0):
            ks.append(k)
    ks = np.pi * np.array(ks, dtype=np.float64)
    amps = rng.standard_normal((n_modes, 3)) / np.sum(ks**2, axis=1)[:, None]
    phases = rng.uniform(0.0, 2 * np.pi, size=n_modes)
    arg = nodes @ ks.T + phases[None, :]  # [n, modes]
    kxa = np.cross(ks, amps)  # [modes, 3]
    return -np.sin(arg) @ kxa


def gaussian_blob(nodes: np.ndarray, center, sigma: float, axis) -> np.ndarray:
    """exp(-|x - center|^2 / sigma^2) times a fixed unit axis."""
    d2 = np.sum((nodes - np.asarray(center)[None, :]) ** 2, axis=1)
    ax = np.asarray(axis, dtype=np.float64)
    ax = ax / np.linalg.norm(ax)
    return np.exp(-d2 / sigma**2)[:, None] * ax[None, :]


def hill_vorticity(nodes: np.ndarray, A=1.0) -> np.ndarray:
    """Hill's spherical vortex: omega = A (-y, x, 0), i.e. omega_theta = A r (linear)."""
    return A * np.stack([-nodes[:, 1], nodes[:, 0], np.zeros(len(nodes))], axis=1)


def hill_velocity(X, A=1.0, a=1.0):
    """Velocity of Hill's spherical vortex in the frame where the fluid is at rest far away.

    From the Stokes stream function psi = (A/10) r^2 (a^2 - r^2 - z^2) inside
    (translation speed U = 2 A a^2 / 15): u_r = A r z / 5,
    u_z = (A/5)(5a^2/3 - 2 r^2 - z^2) inside, a point dipole
    (U a^3 / 2 R^3)(3 (z.R^) R^ - z^) outside.  omega = A (-y, x, 0) inside.
    """
    X = np.asarray(X, dtype=np.float64)
    x, y, z = X.T
    r = np.hypot(x, y)
    R = np.linalg.norm(X, axis=1)
    U = 2.0 * A * a * a / 15.0
    ur = A * r * z / 5.0
    uz = A / 5.0 * (5.0 * a * a / 3.0 - 2.0 * r * r - z * z)
    safe = np.where(r > 0, r, 1.0)
    vin = np.stack([ur * x / safe, ur * y / safe, uz], axis=1)
    Rs = np.where(R > 0, R, 1.0)
    rh = X / Rs[:, None]
    vout = U * a**3 / (2.0 * Rs[:, None] ** 3) * (3.0 * rh[:, 2:3] * rh - np.array([0.0, 0.0, 1.0]))
    return np.where((R < a)[:, None], vin, vout)
