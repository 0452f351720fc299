"""Pins of the rotation diagnostic and the adaptivity map (``oracle/diagnostics.py``)
against closed forms: a grain rotated by theta (Eq. amprot) has omega = sin(theta)
exactly; omega ignores global phases and uniform displacements; the map of
Eq. hhh takes its three branches where the construction says."""
import numpy as np
import pytest

import oracle as O
from oracle import diagnostics as D
from paper_1902_09761_gb300 import inputs


@pytest.mark.parametrize("theta_deg", [-12.0, -3.0, 0.0, 2.5, 9.0])
def test_uniform_rotated_hex_grain_has_omega_sin_theta(theta_deg):
    k = O.hex_k()
    shape, h = (48, 64), (np.pi / 2, np.pi / 2)
    phi = 0.2
    owner = np.zeros(shape, dtype=int)
    eta = inputs.grain_state(k, phi, shape, h, [[0.0, 0.0]], [np.deg2rad(theta_deg)], owner)
    om = D.rotation_field(eta, k, h)
    # the grid is not periodic for the rotated wave: test away from the wrap-around
    inner = om[0][2:-2, 2:-2]
    assert np.max(np.abs(inner - np.sin(np.deg2rad(theta_deg)))) <= 1e-12


def test_rotated_bcc_grain_about_z_has_only_omega_12():
    k = O.bcc_k()
    shape, h = (12, 14, 16), (np.pi / 2,) * 3
    th = np.deg2rad(8.0)
    eta = inputs.grain_state(k, 0.15, shape, h, [[0.0, 0.0, 0.0]], [th], np.zeros(shape, dtype=int))
    om = D.rotation_field(eta, k, h)[:, 2:-2, 2:-2, 2:-2]
    assert np.max(np.abs(om[0])) <= 1e-12 and np.max(np.abs(om[1])) <= 1e-12
    assert np.max(np.abs(om[2] - np.sin(th))) <= 1e-12


def test_omega_ignores_global_phase_and_uniform_displacement():
    k = O.hex_k()
    shape, h = (40, 40), (np.pi / 2, np.pi / 2)
    eta = inputs.single_grain(k, 0.2, shape, h, 20.0, 6.0, seed=1, noise=1e-3)
    u0 = np.array([0.7, -1.3])
    shifted = eta * np.exp(1j * (k @ u0))[:, None, None] * np.exp(0.4j)
    a = D.rotation_field(eta, k, h)
    b = D.rotation_field(shifted, k, h)
    assert np.max(np.abs(a - b)) <= 1e-12


def test_adaptivity_map_branches():
    k = O.hex_k()
    shape, h = (96, 96), (np.pi / 2, np.pi / 2)
    th = 7.0
    eta = inputs.single_grain(k, 0.2, shape, h, 40.0, th, seed=2, noise=0.0)
    n, h_int, h_max, eps, A_min = 10.0, 1.0, 40.0, 0.02, 0.05
    hm = D.adaptivity_map(eta, k, h, n, h_int, h_max, eps, A_min)
    A = D.amplitude_A(eta)
    gA = D.grad_norm(A, h)
    # liquid: h_max; interface band: h_int; grain interior: the rotation bound
    assert np.all(hm[(A <= A_min) & (gA < eps)] == h_max)
    assert np.all(hm[gA >= eps] == h_int)
    interior = (A > A_min) & (gA < eps)
    interior[0:4, :] = interior[-4:, :] = interior[:, 0:4] = interior[:, -4:] = False
    s = np.sin(0.5 * np.arcsin(np.sin(np.deg2rad(th))))
    expect = min(max(np.pi / (n * 1.0 * s), h_int), h_max)
    assert interior.sum() > 100
    assert np.max(np.abs(hm[interior] - expect)) <= 1e-9 * expect
