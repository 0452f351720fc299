"""Pins of the Picard / Jacobian oracle (``oracle/picard.py``): the sparse
stencil matrices against the FFT-diagonal operator, the Jacobian diagonal
against central differences of N in direction eta_j, K = 1 without the
Jacobian against the explicit step, and converged iterations against the
residual of the fully implicit backward Euler step (with and without the
Jacobian, which must reach the same point, the Jacobian faster)."""
import numpy as np
import pytest

import oracle as O
from oracle import picard as PC
from paper_1902_09761_gb300 import inputs

P = O.params_from_paper(0.98, 0.01, 0.25, 0.5)


def _rand(shape, seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return scale * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))


@pytest.mark.parametrize("shape,h", [((6, 8), (1.1, 0.9)), ((4, 5, 6), (1.1, 0.9, 1.2))])
def test_sparse_G_equals_stencil(shape, h):
    kj = np.array([0.3, -0.8, 0.5][: len(h)])
    u = _rand(shape, 1)
    G = PC.g_matrix(kj, shape, h)
    assert np.max(np.abs((G @ u.ravel()).reshape(shape) - O.apply_G(u, kj, h))) <= 1e-13


@pytest.mark.parametrize("kind", ["hex", "bcc"])
def test_jacobian_diag_is_holomorphic_derivative(kind):
    L = O.hex_lattice() if kind == "hex" else O.bcc_lattice()
    shape = (L.J, 5, 6) if kind == "hex" else (L.J, 3, 4, 3)
    eta = _rand(shape, 2)
    D = PC.jacobian_diag(eta, P, L)
    eps = 1e-6
    for j in range(L.J):
        e_re = np.zeros(shape, complex)
        e_re[j] = eps
        dN_dx = (L.nonlinear(eta + e_re, P)[j] - L.nonlinear(eta - e_re, P)[j]) / (2 * eps)
        dN_dy = (L.nonlinear(eta + 1j * e_re, P)[j] - L.nonlinear(eta - 1j * e_re, P)[j]) / (2 * eps)
        ref = 0.5 * (dN_dx - 1j * dN_dy)  # d/d eta = (d/dx - i d/dy) / 2
        assert np.max(np.abs(D[j] - ref)) <= 1e-7 * max(1.0, np.max(np.abs(ref)))
        assert np.max(np.abs(D[j].imag)) <= 1e-12 * max(1.0, np.max(np.abs(D[j])))


def test_hex_jacobian_closed_form_equals_table():
    L = O.hex_lattice()
    eta = _rand((3, 6, 7), 3)
    a = PC.jacobian_diag_hex(eta, P)
    b = PC.jacobian_diag_table(eta, P, L.table)
    assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(a))


def test_single_iteration_without_jacobian_is_the_explicit_step():
    L, h = O.hex_lattice(), (np.pi / 2, np.pi / 2)
    eta = O.uniform_solid_hex(P) + _rand((3, 12, 10), 4, 0.05)
    a, _ = PC.step_picard(eta, 0.7, P, L, h, 1, jacobian=False)
    b, _ = O.step(eta, 0.7, P, L, h)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))


@pytest.mark.parametrize("kind", ["hex", "bcc"])
def test_converged_iterations_solve_backward_euler(kind):
    L = O.hex_lattice() if kind == "hex" else O.bcc_lattice()
    if kind == "hex":
        shape, h = (16, 20), (np.pi / 2, np.pi / 2)
        eta = inputs.single_grain(L.k, O.uniform_solid_hex(P), shape, h, 8.0, 6.0, seed=5, noise=1e-2)
    else:
        shape, h = (6, 6, 8), (np.pi / 2,) * 3
        eta = O.uniform_solid_bcc(P) + _rand((6,) + shape, 5, 0.02)
    dt = 1.0
    scale = np.max(np.abs(eta)) / dt
    res = {}
    for jac in (True, False):
        errs = []
        for K in (2, 4, 8, 16):
            e, _ = PC.step_picard(eta, dt, P, L, h, K, jacobian=jac)
            errs.append(np.max(np.abs(PC.backward_euler_residual(e, eta, dt, P, L, h))) / scale)
        res[jac] = (errs, e)
        assert errs[3] < errs[2] < errs[1] < errs[0]  # the iteration contracts (linearly)
    assert res[True][0][3] <= 1e-11
    assert res[True][0][2] < res[False][0][2]  # the Jacobian speeds it up
    K = 40
    e_plain, _ = PC.step_picard(eta, dt, P, L, h, K, jacobian=False)
    assert np.max(np.abs(e_plain - res[True][1])) <= 1e-9 * np.max(np.abs(e_plain))
