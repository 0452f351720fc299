"""Seeded synthetic initial states shaped like the paper's polycrystal setups.

This module holds no arithmetic of the time step: it only lays out initial
amplitudes.  The lattice vectors ``k`` and the relaxed-solid amplitude ``phi``
are arguments, so the same arrays can be handed to the CUDA library and to any
checker.

Recipe (Sec. II.D, Eq. amprot, and the setups of Sec. III):

* node-centred periodic grid, node i at r = i h;
* a grain rotated by theta has eta_j = phi exp(i dk_j . (r - c)), with
  dk_j = R(theta) k_j - k_j, R the counter-clockwise rotation (in 3D about the
  z axis, i.e. [001]) and c the grain centre;
* noise: real and imaginary parts i.i.d. normal with standard deviation
  ``noise`` at every point and amplitude, from ``numpy.random.default_rng(seed)``;
* Voronoi grains use the periodic minimum-image distance to seeded centres.
"""
from __future__ import annotations

import numpy as np


def grid_coords(shape, h):
    """Node coordinates (x, y[, z]) broadcastable to ``shape`` (array order z, y, x)."""
    dim = len(shape)
    out = []
    for d in range(dim):
        n = shape[dim - 1 - d]
        view = [1] * dim
        view[dim - 1 - d] = n
        out.append((np.arange(n, dtype=float) * h[d]).reshape(view))
    return out


def rotation_matrix(theta_rad: float, dim: int) -> np.ndarray:
    """Counter-clockwise rotation by theta in the x-y plane (about [001] in 3D)."""
    c, s = np.cos(theta_rad), np.sin(theta_rad)
    R = np.eye(dim)
    R[0, 0], R[0, 1], R[1, 0], R[1, 1] = c, -s, s, c
    return R


def delta_k(k, theta_rad: float) -> np.ndarray:
    """dk_j = R(theta) k_j - k_j for every lattice vector."""
    k = np.asarray(k, dtype=float)
    R = rotation_matrix(theta_rad, k.shape[1])
    return k @ R.T - k


def _min_image(x, c, L):
    d = x - c
    return d - L * np.round(d / L)


def add_noise(eta: np.ndarray, rng: np.random.Generator, noise: float) -> np.ndarray:
    if noise > 0:
        eta += noise * (rng.standard_normal(eta.shape) + 1j * rng.standard_normal(eta.shape))
    return eta


def grain_state(k, phi, shape, h, centres, thetas_rad, owner, background=None) -> np.ndarray:
    """eta_j = phi exp(i dk_j(theta_g).(r - c_g)) wherever ``owner == g``.

    ``owner`` is an int array over the grid (-1 = background); ``background``
    is None for liquid (eta = 0) or a real value for an unrotated solid.
    """
    k = np.asarray(k, dtype=float)
    J, dim = k.shape
    coords = grid_coords(shape, h)
    centres = np.asarray(centres, dtype=float).reshape(len(thetas_rad), dim)
    dk = np.stack([delta_k(k, th) for th in thetas_rad])  # (G, J, dim)
    inside = owner >= 0
    g = np.where(inside, owner, 0)
    eta = np.empty((J,) + tuple(shape), dtype=np.complex128)
    for j in range(J):
        ph = np.zeros(shape)
        for d in range(dim):
            ph += dk[g, j, d] * (coords[d] - centres[g, d])
        val = phi * np.exp(1j * ph)
        eta[j] = np.where(inside, val, 0.0 if background is None else background)
    return eta


def single_grain(k, phi, shape, h, radius, theta_deg, seed=0, noise=1e-3, matrix=None):
    """One circular/spherical grain of ``radius`` at the domain centre.

    Outside the grain: liquid (``matrix=None``) or an unrotated solid of
    amplitude ``matrix``.
    """
    dim = len(shape)
    L = [shape[dim - 1 - d] * h[d] for d in range(dim)]
    c = [0.5 * L[d] for d in range(dim)]
    coords = grid_coords(shape, h)
    r2 = np.zeros(shape)
    for d in range(dim):
        r2 = r2 + (coords[d] - c[d]) ** 2
    owner = np.where(r2 <= radius * radius, 0, -1)
    eta = grain_state(k, phi, shape, h, [c], [np.deg2rad(theta_deg)], owner, background=matrix)
    return add_noise(eta, np.random.default_rng(seed), noise)


def voronoi_grains(k, phi, shape, h, ngrains, theta_max_deg, seed=1, noise=1e-3):
    """``ngrains`` Voronoi grains filling the periodic box, rotations U[-max, max] deg."""
    dim = len(shape)
    rng = np.random.default_rng(seed)
    L = np.array([shape[dim - 1 - d] * h[d] for d in range(dim)])
    centres = rng.uniform(0.0, 1.0, size=(ngrains, dim)) * L
    thetas = np.deg2rad(rng.uniform(-theta_max_deg, theta_max_deg, size=ngrains))
    coords = grid_coords(shape, h)
    best = np.full(shape, np.inf)
    owner = np.zeros(shape, dtype=np.int64)
    for g in range(ngrains):
        d2 = np.zeros(shape)
        for d in range(dim):
            d2 = d2 + _min_image(coords[d], centres[g, d], L[d]) ** 2
        closer = d2 < best
        best = np.where(closer, d2, best)
        owner = np.where(closer, g, owner)
    eta = grain_state(k, phi, shape, h, centres, thetas, owner)
    return add_noise(eta, rng, noise)


def random_amplitudes(J, shape, seed=0, scale=0.1) -> np.ndarray:
    """Random complex amplitudes (for operator-level parity cases)."""
    rng = np.random.default_rng(seed)
    return scale * (rng.standard_normal((J,) + tuple(shape)) + 1j * rng.standard_normal((J,) + tuple(shape)))


def hex_vectors() -> np.ndarray:
    """Triangular-lattice reciprocal vectors as input data (Sec. II)."""
    s3 = np.sqrt(3.0)
    return np.array([[-s3 / 2, -0.5], [0.0, 1.0], [s3 / 2, -0.5]])


def bcc_vectors() -> np.ndarray:
    """bcc <110>/sqrt(2) reciprocal vectors as input data."""
    r = 1.0 / np.sqrt(2.0)
    return r * np.array([[1, 1, 0], [1, -1, 0], [1, 0, 1], [1, 0, -1], [0, 1, 1], [0, 1, -1]], dtype=float)


# Workloads (sizes and recipes of the configurations this library is measured on)
HEX_H = np.pi / 2


def hex_grain_128(phi):
    """2D hexagonal, 128x128, h = pi/2, grain R = 30 rotated 5 deg in liquid, noise 1e-3, seed 0."""
    return single_grain(hex_vectors(), phi, (128, 128), (HEX_H, HEX_H), 30.0, 5.0, seed=0, noise=1e-3)


def hex_voronoi(phi, n=4096, ngrains=16, seed=1):
    """2D hexagonal, n x n, h = pi/2, 16 Voronoi grains, rotations U[-10,10] deg, noise 1e-3."""
    return voronoi_grains(hex_vectors(), phi, (n, n), (HEX_H, HEX_H), ngrains, 10.0, seed=seed, noise=1e-3)


def bcc_sphere(phi, n=256, radius=60.0, seed=2):
    """3D bcc, n^3, h = pi/2, sphere R = 60 rotated 8 deg about [001] in an unrotated matrix."""
    h = (HEX_H,) * 3
    return single_grain(bcc_vectors(), phi, (n, n, n), h, radius, 8.0, seed=seed, noise=1e-3, matrix=phi)


def batch_spec(nruns=64, sizes=(128, 256, 512, 1024), theta_max_deg=10.0, seed=7):
    """Independent 2D hexagonal runs: grid size N drawn uniformly from ``sizes``
    (N x N), grain rotation U[-max, max] deg, and a noise seed per run.
    Returns a list of (N, theta_deg, noise_seed)."""
    rng = np.random.default_rng(seed)
    ns = rng.choice(np.asarray(sizes), size=nruns)
    th = rng.uniform(-theta_max_deg, theta_max_deg, size=nruns)
    return [(int(ns[r]), float(th[r]), int(seed * 100003 + r)) for r in range(nruns)]


def batch_run_state(phi, n, theta_deg, noise_seed, shape=None):
    """One run of a batch: a circular grain of radius n h / 4 (a fifth of the box
    area) rotated ``theta_deg`` in liquid at the centre of an n x n hexagonal box
    (or of ``shape``), h = pi/2, noise 1e-3."""
    shape = (n, n) if shape is None else tuple(shape)
    radius = 0.25 * min(shape) * HEX_H
    return single_grain(hex_vectors(), phi, shape, (HEX_H, HEX_H), radius, theta_deg, seed=noise_seed, noise=1e-3)
