"""Plain FP64 oracle of the rotation-field diagnostic and the adaptivity map.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. II.D (Eqs. amprot, rot, hhh).  The local displacement u solves
k_j . u = theta_j, theta_j the phase of eta_j, and the rotation tensor is
omega_il = 1/2 (du_i/dx_l - du_l/dx_i).  Readings (the paper cites, but does
not print, the explicit inversion):

* phase gradients are central differences of the unwrapped phase,
  d theta_j/dx_d = arg(eta_j(r + h e_d) conj(eta_j(r - h e_d))) / (2 h_d),
  exact for a plane wave exp(i dk . r) while |dk_d| h_d < pi/2;
* u is the least-squares solution of the J equations k_j . u = theta_j,
  u = M^{-1} sum_j k_j theta_j with M = sum_j k_j k_j^T, so that
  du_i/dx_l = sum_j (M^{-1} k_j)_i d theta_j/dx_l;
* omega is reported as (omega_12) in 2D and (omega_23, omega_31, omega_12)
  in 3D (rotation about x, y, z); a grain rotated counter-clockwise by theta
  about z has omega_12 = sin(theta) exactly;
* where some |eta_j|^2 is below ``amp_floor`` the phase is undefined and
  omega is set to 0 (the liquid; the paper calls omega ill-posed there);
* A = sqrt(2 sum_j |eta_j|^2), grad A by central differences;
* in Eq. hhh the rotation angle is theta = asin(min(max_d |omega_d|, 1)) and
  lambda_j(theta) = 2 pi / |dk_j(theta)| with |dk_j(theta)| = 2 |k_j| sin(theta/2)
  (the largest over rotation axes), so h_amp = pi / (n max_j |k_j| sin(theta/2));
  theta = 0 gives h_amp = infinity.  "A > 0" is read as A > A_min.
"""
from __future__ import annotations

import numpy as np


def _shift(u, d, s, dim):
    """u at r + s h e_d on the periodic grid (axis of x is the last)."""
    return np.roll(u, -s, axis=u.ndim - 1 - d)


def phase_gradients(eta, h):
    """d theta_j / dx_d for every j, d: shape (J, dim) + grid."""
    dim = len(h)
    out = np.empty((eta.shape[0], dim) + eta.shape[1:])
    for j in range(eta.shape[0]):
        for d in range(dim):
            p = _shift(eta[j], d, 1, dim)
            m = _shift(eta[j], d, -1, dim)
            out[j, d] = np.angle(p * np.conj(m)) / (2.0 * h[d])
    return out


def rotation_field(eta, k, h, amp_floor=1e-12):
    """omega: (1,) + grid in 2D (omega_12), (3,) + grid in 3D (omega_23, omega_31, omega_12)."""
    k = np.asarray(k, dtype=float)
    J, dim = k.shape
    M = sum(np.outer(k[j], k[j]) for j in range(J))
    W = np.linalg.solve(M, k.T).T  # W_j = M^{-1} k_j
    g = phase_gradients(eta, h)
    du = np.zeros((dim, dim) + eta.shape[1:])
    for i in range(dim):
        for l in range(dim):
            du[i, l] = sum(W[j, i] * g[j, l] for j in range(J))

    def om(i, l):
        return 0.5 * (du[i, l] - du[l, i])

    omega = np.stack([om(0, 1)]) if dim == 2 else np.stack([om(1, 2), om(2, 0), om(0, 1)])
    ok = np.all(np.abs(eta) ** 2 >= amp_floor, axis=0)
    return np.where(ok, omega, 0.0)


def amplitude_A(eta):
    return np.sqrt(2.0 * np.sum(np.abs(eta) ** 2, axis=0))


def grad_norm(f, h):
    dim = len(h)
    s = np.zeros_like(f)
    for d in range(dim):
        g = (_shift(f, d, 1, dim) - _shift(f, d, -1, dim)) / (2.0 * h[d])
        s = s + g * g
    return np.sqrt(s)


def adaptivity_map(eta, k, h, n, h_int, h_max, eps, A_min, amp_floor=1e-12):
    """The local grid size h of Eq. hhh at every point."""
    k = np.asarray(k, dtype=float)
    omega = rotation_field(eta, k, h, amp_floor)
    A = amplitude_A(eta)
    gA = grad_norm(A, h)
    wmax = np.max(np.abs(omega), axis=0)
    theta = np.arcsin(np.minimum(wmax, 1.0))
    kmax = float(np.max(np.linalg.norm(k, axis=1)))
    s = np.sin(0.5 * theta)
    with np.errstate(divide="ignore"):
        h_amp = np.where(s > 0.0, np.pi / (n * kmax * np.where(s > 0.0, s, 1.0)), np.inf)
    grain = np.minimum(np.maximum(h_amp, h_int), h_max)
    return np.where(gA >= eps, h_int, np.where(A > A_min, grain, h_max))
