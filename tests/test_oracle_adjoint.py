"""Pins of the oracle's adjoint (``oracle/adjoint.py``) against what the
mathematics fixes: central finite differences of the oracle's own forward map
(the definition of the derivative), the closed-form triangular derivatives
against the resonance-table ones (two independent derivations), and, with
t = v = 0 (N = 0), the Fourier closed form of the gradient of the misfit.
"""
from dataclasses import replace

import numpy as np
import pytest

import oracle as O

P = O.params_from_paper(0.98, 0.01, 0.25, 0.5)


def _rand(shape, seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return scale * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))


def _lat(kind):
    return O.hex_lattice() if kind == "hex" else O.bcc_lattice()


def _shape(kind):
    return (3, 10, 12) if kind == "hex" else (6, 5, 6, 4)


def _h(kind):
    return (1.1, 0.9) if kind == "hex" else (1.1, 0.9, 1.2)


def _re_dot(a, b):
    return float(np.sum(np.conj(a) * b).real)


@pytest.mark.parametrize("kind", ["hex", "bcc"])
def test_nonlinear_vjp_matches_finite_difference(kind):
    L = _lat(kind)
    eta, w, d = _rand(_shape(kind), 1), _rand(_shape(kind), 2), _rand(_shape(kind), 3)
    vjp = O.nonlinear_vjp(eta, w, P, L)
    eps = 1e-6
    fd = (_re_dot(w, L.nonlinear(eta + eps * d, P)) - _re_dot(w, L.nonlinear(eta - eps * d, P))) / (2 * eps)
    assert _re_dot(vjp, d) == pytest.approx(fd, rel=1e-8)


def test_hex_closed_form_vjp_equals_table_vjp():
    L = O.hex_lattice()
    eta, w = _rand((3, 7, 9), 4), _rand((3, 7, 9), 5)
    a = O.nonlinear_vjp_hex(eta, w, P)
    b = O.nonlinear_vjp_table(eta, w, P, L.table)
    assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(a))


@pytest.mark.parametrize("kind", ["hex", "bcc"])
def test_step_adjoint_matches_finite_difference(kind):
    L, h, dt = _lat(kind), _h(kind), 0.7
    eta, lam, d = _rand(_shape(kind), 6), _rand(_shape(kind), 7), _rand(_shape(kind), 8)
    eta1, _ = O.step(eta, dt, P, L, h)
    lam_n, d_dB = O.step_adjoint(eta, eta1, lam, dt, P, L, h)
    eps = 1e-6
    f = lambda e, q=P: _re_dot(lam, O.step(e, dt, q, L, h)[0])  # noqa: E731
    fd = (f(eta + eps * d) - f(eta - eps * d)) / (2 * eps)
    assert _re_dot(lam_n, d) == pytest.approx(fd, rel=1e-8)
    fd_dB = (f(eta, replace(P, dB=P.dB + eps)) - f(eta, replace(P, dB=P.dB - eps))) / (2 * eps)
    assert d_dB == pytest.approx(fd_dB, rel=1e-7)


@pytest.mark.parametrize("w_energy", [0.0, 1.0])
def test_rollout_gradient_matches_central_differences(w_energy):
    L, h, dt, K = O.hex_lattice(), (np.pi / 2, np.pi / 2), 1.0, 5
    shape = (3, 12, 16)
    phi = O.uniform_solid_hex(P)
    eta0 = phi + _rand(shape, 9, 0.05)
    target = _rand(shape, 10, 0.1)
    g, g_dB = O.rollout_gradient(eta0, P.dB, target, dt, K, P, L, h, w_energy)
    eps = 1e-6
    loss = lambda e, dB=P.dB: O.rollout_loss(e, dB, target, dt, K, P, L, h, w_energy)  # noqa: E731
    rng = np.random.default_rng(11)
    for _ in range(4):
        d = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
        fd = (loss(eta0 + eps * d) - loss(eta0 - eps * d)) / (2 * eps)
        assert _re_dot(g, d) == pytest.approx(fd, rel=1e-6, abs=1e-9)
    fd_dB = (loss(eta0, P.dB + eps) - loss(eta0, P.dB - eps)) / (2 * eps)
    assert g_dB == pytest.approx(fd_dB, rel=1e-6)


def test_linear_case_gradient_equals_fourier_closed_form():
    # t = v = 0: N = 0 and eta^K_j = (S_j^{-1}/dt)^K eta0_j, with S_j Hermitian, so the
    # gradient of 1/2 h^d |eta^K|^2 is h^d (S_j^{-1}/dt)^{2K} eta0_j, diagonal in Fourier space.
    q = replace(P, t=0.0, v=0.0)
    L, h, dt, K = O.hex_lattice(), (0.8, 1.3), 0.5, 4
    shape = (3, 8, 10)
    eta0 = _rand(shape, 12)
    g, _ = O.rollout_gradient(eta0, q.dB, np.zeros(shape), dt, K, q, L, h, w_energy=0.0)
    vol = h[0] * h[1]
    for j in range(3):
        s = O.schur_symbol(L.k[j], dt, q, shape[1:], h)
        closed = np.fft.ifft2(np.fft.fft2(eta0[j]) * (1.0 / (dt * s)) ** (2 * K)) * vol
        assert np.max(np.abs(g[j] - closed)) <= 1e-12 * np.max(np.abs(closed))
