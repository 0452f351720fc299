"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test names what fixes the expected value: a number printed in the paper
(``tests/golden/paper_constants.json``), a closed form derived from the model,
a dense direct solve, a brute-force cell average, the continuum operator, or
an invariance of the equations.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_1902_09761_gb300 import inputs

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
P = O.params_from_paper(**{k: v for k, v in GOLD["energy_parameters"].items() if not k.startswith("_")})
H2 = (np.pi / 2, np.pi / 2)


def test_parameter_mapping_matches_standard_set():
    # Sec. II prints a0..a3; the standard set used for the configs is dB=0.02, Bx=0.98, t=0.5, v=1/3.
    assert P.dB == pytest.approx(0.02, abs=1e-15)
    assert P.Bx == pytest.approx(0.98, abs=1e-15)
    assert P.t == pytest.approx(0.5, abs=1e-15)
    assert P.v == pytest.approx(1.0 / 3.0, abs=1e-15)


def test_lattice_vectors():
    np.testing.assert_allclose(O.hex_k(), np.array(GOLD["triangular_k"]["k"]), atol=1e-15)
    for k in (O.hex_k(), O.bcc_k()):
        np.testing.assert_allclose(O.kappa(k), 1.0, atol=1e-15)
    np.testing.assert_allclose(O.hex_k().sum(axis=0), 0.0, atol=1e-15)


# --- finite-difference operator ------------------------------------------------


@pytest.mark.parametrize("shape,h", [((12, 10), (0.7, 0.9)), ((6, 8, 10), (0.5, 0.6, 0.8))])
def test_symbol_equals_stencil_on_grid_modes(shape, h):
    # G_h applied to every grid Fourier mode returns the mode times symbol_G (exact).
    dim = len(h)
    k = O.hex_k()[1] if dim == 2 else O.bcc_k()[2]
    coords = inputs.grid_coords(shape, h)
    g = O.symbol_G(k, shape, h)
    rng = np.random.default_rng(3)
    for _ in range(6):
        m = [rng.integers(0, shape[dim - 1 - d]) for d in range(dim)]
        q = [2 * np.pi * m[d] / (shape[dim - 1 - d] * h[d]) for d in range(dim)]
        w = np.exp(1j * sum(q[d] * coords[d] for d in range(dim)))
        idx = tuple(m[dim - 1 - a] for a in range(dim))
        np.testing.assert_allclose(O.apply_G(w, k, h), g[idx] * w, atol=1e-11)


def test_stencil_converges_to_continuum_operator_second_order():
    # G = Delta + 2i k.grad (Sec. II): on e^{iq.r}, G gives (-|q|^2 - 2 k.q) e^{iq.r}.
    k = O.hex_k()[0]
    q = np.array([0.3, -0.2])
    errs = []
    for h in (0.2, 0.1, 0.05):
        n = 64
        coords = inputs.grid_coords((n, n), (h, h))
        w = np.exp(1j * (q[0] * coords[0] + q[1] * coords[1]))
        # only interior points matter for the local truncation error; the wave is not periodic
        got = O.apply_G(w, k, (h, h))[5:-5, 5:-5]
        exact = (-(q @ q) - 2 * (k @ q)) * w[5:-5, 5:-5]
        errs.append(np.max(np.abs(got - exact)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.6 < r1 < 4.4 and 3.6 < r2 < 4.4


def test_G_hermitian_and_annihilates_constants():
    shape, h = (6, 5), (0.8, 1.1)
    for k in O.hex_k():
        G = O.dense_operator(lambda u: O.apply_G(u, k, h), shape)
        np.testing.assert_allclose(G, G.conj().T, atol=1e-13)
        np.testing.assert_allclose(G @ np.ones(G.shape[0]), 0.0, atol=1e-13)


# --- the step -----------------------------------------------------------------


@pytest.mark.parametrize(
    "shape,h,lat",
    [((8, 8), H2, "hex"), ((6, 10), (1.0, 0.8), "hex"), ((4, 4, 4), (np.pi / 2,) * 3, "bcc")],
)
def test_fft_solve_matches_dense_block_lu(shape, h, lat):
    # Dense LU of the assembled 2n x 2n block matrix (Eq. linear_system2, M = I)
    # against the oracle's FFT Schur solve and zeta = G_h eta.
    L = O.hex_lattice() if lat == "hex" else O.bcc_lattice()
    rng = np.random.default_rng(7)
    eta = 0.2 * (rng.standard_normal((L.J,) + shape) + 1j * rng.standard_normal((L.J,) + shape))
    dt = 0.7
    new, zeta = O.step(eta, dt, P, L, h)
    b = O.rhs(eta, dt, P, L)
    n = int(np.prod(shape))
    for j in range(L.J):
        A = O.dense_block_matrix(L.k[j], dt, P, shape, h)
        x = np.linalg.solve(A, np.concatenate([np.zeros(n), b[j].ravel()]))
        np.testing.assert_allclose(x[n:].reshape(shape), new[j], atol=1e-12)
        np.testing.assert_allclose(x[:n].reshape(shape), zeta[j], atol=1e-12)
        # apply_A is the same matrix
        y1, y2 = O.apply_A(zeta[j], new[j], L.k[j], dt, P, h)
        np.testing.assert_allclose(np.concatenate([y1.ravel(), y2.ravel()]), A @ x, atol=1e-12)


@pytest.mark.parametrize("mode", [(0, 0), (1, 0), (3, -2), (8, 8), (-5, 8)])
def test_fourier_mode_decay(mode):
    # With t = v = 0 the step is backward Euler on the linear flow:
    # eta^{n+1} = eta^n / (1 + dt kap (dB + Bx lam^2)) for a mode with G_h w = lam w.
    # lam is measured by applying the stencil, not taken from the symbol formula.
    p = O.Params(dB=P.dB, Bx=P.Bx, t=0.0, v=0.0)
    L = O.hex_lattice()
    shape, h, dt = (16, 16), H2, 1.0
    x, y = inputs.grid_coords(shape, h)
    q = [2 * np.pi * mode[0] / (16 * h[0]), 2 * np.pi * mode[1] / (16 * h[1])]
    w = np.exp(1j * (q[0] * x + q[1] * y))
    eta = np.stack([w, 2 * w, -w])
    new, _ = O.step(eta, dt, p, L, h)
    for j in range(3):
        lam = (O.apply_G(w, L.k[j], h) / w).mean()
        assert abs(lam.imag) < 1e-12
        fac = 1.0 / (1.0 + dt * (p.dB + p.Bx * lam.real ** 2))
        np.testing.assert_allclose(new[j], fac * eta[j], atol=1e-13)


def test_uniform_solid_is_fixed_point_hex():
    # Closed form phi = (t + sqrt(t^2 - 15 v dB)) / (15 v); value 0.1774596669 at the standard set.
    phi = O.uniform_solid_hex(P)
    assert phi == pytest.approx((0.5 + np.sqrt(0.25 - 15 * (1 / 3) * 0.02)) / 5.0, rel=1e-15)
    assert phi == pytest.approx(0.1774596669, abs=1e-10)
    L = O.hex_lattice()
    eta = np.full((3, 8, 8), phi, dtype=complex)
    np.testing.assert_allclose(P.dB * eta + L.nonlinear(eta, P), 0.0, atol=1e-15)
    new, zeta = O.step(eta, 1.0, P, L, H2)
    np.testing.assert_allclose(new, eta, atol=1e-15)
    np.testing.assert_allclose(zeta, 0.0, atol=1e-15)
    # liquid is a fixed point too
    new0, _ = O.step(np.zeros_like(eta), 1.0, P, L, H2)
    assert np.all(new0 == 0)


def test_uniform_solid_is_fixed_point_bcc():
    phi = O.uniform_solid_bcc(P)
    assert phi == pytest.approx(0.1224440020, abs=1e-9)
    L = O.bcc_lattice()
    eta = np.full((6, 4, 4, 4), phi, dtype=complex)
    np.testing.assert_allclose(P.dB * eta + L.nonlinear(eta, P), 0.0, atol=1e-15)
    # the uniform bulk density is 6 dB phi^2 - 16 t phi^3 + 135 v phi^4 (cell-average rule)
    f = L.bulk_density(eta, P)[0, 0, 0]
    assert f == pytest.approx(6 * P.dB * phi**2 - 16 * P.t * phi**3 + 135 * P.v * phi**4, rel=1e-13)


# --- bulk polynomial ------------------------------------------------------------


def _cell_average_bruteforce(k, eta_const, p, cell, m):
    """Mean of dB/2 n^2 - t/3 n^3 + v/4 n^4 over a period cell sampled on m^dim points."""
    dim = len(cell)
    axes = [np.arange(m) * cell[d] / m for d in range(dim)]
    grids = np.meshgrid(*axes, indexing="ij")
    n = np.zeros(grids[0].shape)
    for j in range(len(k)):
        ph = sum(k[j][d] * grids[d] for d in range(dim))
        n = n + 2.0 * (eta_const[j] * np.exp(1j * ph)).real
    f = 0.5 * p.dB * n**2 - p.t / 3.0 * n**3 + 0.25 * p.v * n**4
    return f.mean()


@pytest.mark.parametrize("lat", ["hex", "bcc"])
def test_resonance_table_equals_bruteforce_cell_average(lat):
    # Density Eq. of Sec. II with n0 = 0; sampling is exact for these trigonometric polynomials.
    if lat == "hex":
        L, cell = O.hex_lattice(), (4 * np.pi / np.sqrt(3), 4 * np.pi)
    else:
        L, cell = O.bcc_lattice(), (2 * np.pi * np.sqrt(2),) * 3
    rng = np.random.default_rng(11)
    for _ in range(3):
        e = 0.3 * (rng.standard_normal(L.J) + 1j * rng.standard_normal(L.J))
        brute = _cell_average_bruteforce(L.k, e, P, cell, 24 if lat == "hex" else 12)
        table = O.bulk_density_table(e.reshape((L.J,) + (1,) * L.dim), P, L.table).ravel()[0]
        assert table == pytest.approx(brute, rel=1e-12, abs=1e-14)


def test_hex_closed_form_equals_table():
    L = O.hex_lattice()
    eta = inputs.random_amplitudes(3, (5, 7), seed=5, scale=0.3)
    np.testing.assert_allclose(O.nonlinear_hex(eta, P), O.nonlinear_table(eta, P, L.table), atol=1e-14)
    np.testing.assert_allclose(O.bulk_density_hex(eta, P), O.bulk_density_table(eta, P, L.table), atol=1e-14)


@pytest.mark.parametrize("lat", ["hex", "bcc"])
def test_nonlinear_term_is_wirtinger_derivative_of_bulk(lat):
    # df = 2 Re sum_j conj(df/d conj(eta_j)) d eta_j, with df/d conj(eta_j) = dB eta_j + N_j.
    L = O.hex_lattice() if lat == "hex" else O.bcc_lattice()
    rng = np.random.default_rng(2)
    eta = 0.3 * (rng.standard_normal((L.J, 3)) + 1j * rng.standard_normal((L.J, 3)))
    e = rng.standard_normal((L.J, 3)) + 1j * rng.standard_normal((L.J, 3))
    eps = 1e-6
    fd = (L.bulk_density(eta + eps * e, P) - L.bulk_density(eta - eps * e, P)) / (2 * eps)
    grad = P.dB * eta + L.nonlinear(eta, P)
    an = 2.0 * np.sum((np.conj(grad) * e).real, axis=0)
    np.testing.assert_allclose(fd, an, rtol=1e-7, atol=1e-10)


# --- energy ---------------------------------------------------------------------


def test_energy_gradient_matches_finite_difference():
    L = O.hex_lattice()
    h = H2
    eta = inputs.random_amplitudes(3, (8, 6), seed=9, scale=0.2)
    e = inputs.random_amplitudes(3, (8, 6), seed=10, scale=1.0)
    eps = 1e-6
    fd = (O.energy(eta + eps * e, P, L, h) - O.energy(eta - eps * e, P, L, h)) / (2 * eps)
    g = O.energy_gradient(eta, P, L, h)
    an = 2.0 * np.prod(h) * np.sum((np.conj(g) * e).real)
    assert fd == pytest.approx(an, rel=1e-7)


def test_energy_non_increasing_on_grain_growth():
    # 128x128 grain-in-liquid workload, dt = 1, 20 steps: F must not increase.
    phi = O.uniform_solid_hex(P)
    eta = inputs.hex_grain_128(phi)
    L = O.hex_lattice()
    F = [O.energy(eta, P, L, H2)]
    for _ in range(20):
        eta, _ = O.step(eta, 1.0, P, L, H2)
        F.append(O.energy(eta, P, L, H2))
    assert all(b <= a + 1e-12 * abs(a) for a, b in zip(F, F[1:]))


# --- invariances ----------------------------------------------------------------


def test_step_commutes_with_grid_shift_and_phase():
    L = O.hex_lattice()
    eta = inputs.random_amplitudes(3, (10, 12), seed=4, scale=0.15)
    new, _ = O.step(eta, 1.0, P, L, H2)
    sh = np.roll(eta, (3, -5), axis=(1, 2))
    new_sh, _ = O.step(sh, 1.0, P, L, H2)
    np.testing.assert_allclose(new_sh, np.roll(new, (3, -5), axis=(1, 2)), atol=1e-14)
    th = np.array([0.4, -1.1, 0.7])  # sum zero: the cubic coupling is invariant
    ph = np.exp(1j * th).reshape(3, 1, 1)
    new_ph, _ = O.step(eta * ph, 1.0, P, L, H2)
    np.testing.assert_allclose(new_ph, new * ph, atol=1e-14)


# --- preconditioner ------------------------------------------------------------


def test_paper_symbol_spectrum():
    # Sec. II.B: 1D periodic, J = 0, kappa = tau = 1, k = +-1; symbols G -> -(q^2 + 2 q k), K -> q^2.
    g_ = GOLD["preconditioned_symbol_spectrum"]
    q = np.linspace(-40, 40, 400001)
    lams = []
    for k in (-1.0, 1.0):
        ev = O.symbol_AP_inv_eigs(-(q * q + 2 * q * k), q * q, a=1.0, kt=1.0, inv_tau=1.0)
        ev = np.sort(ev.real, axis=-1)
        # one eigenvalue is identically 1, the other is lambda(q)
        one = np.abs(ev - 1.0).argmin(axis=-1)
        other = ev[np.arange(len(q)), 1 - one]
        assert np.allclose(ev[np.arange(len(q)), one], 1.0, atol=1e-9)
        lams.append(other)
    lam = np.concatenate(lams)
    lmin, lmax = lam.min(), lam.max()
    assert lmin == pytest.approx(g_["lambda_min_approx"], abs=0.0015)
    assert lmax == pytest.approx(g_["lambda_max_approx"], abs=0.005)
    rho = (np.sqrt(lmax / lmin) - 1) / (np.sqrt(lmax / lmin) + 1)
    assert rho == pytest.approx(g_["rho"], abs=5e-4)


@pytest.mark.parametrize("tau_mode", ["fold", "plain"])
def test_preconditioner_inverse_exact_inner(tau_mode):
    L = O.hex_lattice()
    h = H2
    b = inputs.random_amplitudes(2, (8, 10), seed=12, scale=1.0)
    for j in range(3):
        c1, c2 = O.apply_Pinv(b[0], b[1], L.k[j], 0.8, P, h, None, tau_mode)
        r1, r2 = O.apply_P(c1, c2, L.k[j], 0.8, P, h, tau_mode)
        np.testing.assert_allclose(r1, b[0], atol=1e-12)
        np.testing.assert_allclose(r2, b[1], atol=1e-12)


@pytest.mark.parametrize("m", [0, 1, 3, 6])
def test_chebyshev_residual_polynomial(m):
    # For an eigenmode of D with eigenvalue l, Chebyshev acceleration returns
    # (1 - T_{m+1}((theta - l)/delta) / T_{m+1}(theta/delta)) / l times the input.
    h = (0.9, 1.3)
    sD, mu = 1.1, 0.95
    lmin, lmax = O.chebyshev_bounds(sD, mu, h)
    theta, delta = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
    x, y = inputs.grid_coords((12, 10), h)
    for mode in [(0, 0), (1, 2), (5, 6), (3, -4)]:
        w = np.exp(1j * (2 * np.pi * mode[0] / (10 * h[0]) * x + 2 * np.pi * mode[1] / (12 * h[1]) * y))
        lam = (O.apply_D(w, sD, mu, h) / w).mean().real
        T = np.polynomial.chebyshev.Chebyshev.basis(m + 1)
        expect = (1.0 - T((theta - lam) / delta) / T(theta / delta)) / lam
        got = O.solve_D_chebyshev(w, sD, mu, h, m)
        np.testing.assert_allclose(got, expect * w, atol=1e-13)


def test_chebyshev_preconditioner_tends_to_exact():
    L = O.hex_lattice()
    b = inputs.random_amplitudes(2, (8, 8), seed=13, scale=1.0)
    ex = O.apply_Pinv(b[0], b[1], L.k[0], 1.0, P, H2, None)
    errs = []
    for m in (2, 6, 12, 30):
        ap = O.apply_Pinv(b[0], b[1], L.k[0], 1.0, P, H2, m)
        errs.append(max(np.abs(ap[0] - ex[0]).max(), np.abs(ap[1] - ex[1]).max()))
    assert errs[-1] < 1e-12 and all(b < a for a, b in zip(errs, errs[1:]))


# --- the preconditioner against the paper's P on grid Fourier modes -------------
#
# Sec. II.B, Eq. preconditioner with M = I:
#   P = [[I, 0], [kt G, D]] [[I, -K], [0, D]],   D = (1/sqrt(tau)) I + sqrt(kt) K,
# where kt = |k_j|^2 Bx is the factor of G in the (2,1) block of A_j and
# 1/tau = 1/dt + |k_j|^2 dB (tau_mode 'fold') or 1/dt ('plain').  Every block
# is a translation-invariant stencil, so P acts on the grid mode e^{iq.r} as a
# 2x2 matrix built from the scalar symbols of K = -L_h and G_h.  The symbols
# below are the textbook ones of the 2d+1-point Laplacian and of the central
# difference, and the coefficients come from the paper's formula, so none of
# ``precond_coeffs``, ``apply_P`` or ``apply_Pinv`` enters the expected values.


def _mode_symbols(kj, shape, h):
    """(kK, g) at the FFT frequencies of ``shape``: K = -L_h and G_h = L_h + 2i k.D_h."""
    dim = len(h)
    kK = np.zeros(shape)
    sk = np.zeros(shape)
    for d in range(dim):
        n = shape[dim - 1 - d]
        q = 2 * np.pi * np.fft.fftfreq(n, d=h[d])
        view = [1] * dim
        view[dim - 1 - d] = n
        q = q.reshape(view)
        kK = kK + (2.0 - 2.0 * np.cos(q * h[d])) / (h[d] * h[d])
        sk = sk + kj[d] * np.sin(q * h[d]) / h[d]
    return kK, -kK - 2.0 * sk


def _paper_P_symbol(kj, dt, p, shape, h, tau_mode):
    kap = float(np.dot(kj, kj))
    kt = kap * p.Bx
    inv_tau = 1.0 / dt + (kap * p.dB if tau_mode == "fold" else 0.0)
    kK, g = _mode_symbols(kj, shape, h)
    dq = np.sqrt(inv_tau) + np.sqrt(kt) * kK
    L = np.zeros(shape + (2, 2))
    L[..., 0, 0] = 1.0
    L[..., 1, 0] = kt * g
    L[..., 1, 1] = dq
    U = np.zeros(shape + (2, 2))
    U[..., 0, 0] = 1.0
    U[..., 0, 1] = -kK
    U[..., 1, 1] = dq
    return L @ U, dict(kt=kt, sD=np.sqrt(inv_tau), mu=np.sqrt(kt), kK=kK, g=g, dq=dq)


def _block_symbol(apply2, shape):
    """2x2 symbol of a translation-invariant block map: column b is the FFT of
    its response to a unit impulse in block b (the response to e^{iq.r} is
    e^{iq.r} times that FFT at q, numpy's sign convention)."""
    dim = len(shape)
    delta = np.zeros(shape, dtype=complex)
    delta[(0,) * dim] = 1.0
    zero = np.zeros(shape, dtype=complex)
    S = np.empty(shape + (2, 2), dtype=complex)
    for b, inp in enumerate(((delta, zero), (zero, delta))):
        out = apply2(*inp)
        for a in range(2):
            S[..., a, b] = np.fft.fftn(out[a])
    return S


# Bx = 0.98 makes kt != sqrt(kt); the second set (dB = 0.3, dt = 0.7) separates
# the two tau modes and 1/tau from 1/dt.
_P_CASES = [
    ("hex", 0, P, 1.0),
    ("hex", 1, P, 1.0),
    ("hex", 2, O.Params(dB=0.3, Bx=0.98, t=0.5, v=1 / 3), 0.7),
    ("bcc", 3, O.Params(dB=0.3, Bx=0.6, t=0.5, v=1 / 3), 0.7),
]


def _case_grid(lat):
    if lat == "hex":
        return O.hex_k(), (10, 12), (np.pi / 2, 1.1)
    return O.bcc_k(), (6, 5, 8), (np.pi / 2, 1.1, 0.9)


@pytest.mark.parametrize("tau_mode", ["fold", "plain"])
@pytest.mark.parametrize("lat,j,p,dt", _P_CASES)
def test_apply_P_equals_paper_symbol(lat, j, p, dt, tau_mode):
    ks, shape, h = _case_grid(lat)
    want, _ = _paper_P_symbol(ks[j], dt, p, shape, h, tau_mode)
    got = _block_symbol(lambda a, b: O.apply_P(a, b, ks[j], dt, p, h, tau_mode), shape)
    np.testing.assert_allclose(got, want, atol=1e-12 * np.abs(want).max())


@pytest.mark.parametrize("tau_mode", ["fold", "plain"])
@pytest.mark.parametrize("lat,j,p,dt", _P_CASES)
def test_apply_Pinv_exact_equals_inverse_of_paper_symbol(lat, j, p, dt, tau_mode):
    ks, shape, h = _case_grid(lat)
    Pq, _ = _paper_P_symbol(ks[j], dt, p, shape, h, tau_mode)
    want = np.linalg.inv(Pq)
    got = _block_symbol(lambda a, b: O.apply_Pinv(a, b, ks[j], dt, p, h, None, tau_mode), shape)
    np.testing.assert_allclose(got, want, atol=1e-12 * np.abs(want).max())


@pytest.mark.parametrize("m", [0, 1, 3])
@pytest.mark.parametrize("lat,j,p,dt", _P_CASES[1:])
def test_apply_Pinv_chebyshev_equals_four_steps_on_symbol(lat, j, p, dt, m):
    # The four steps of Sec. II.B on one mode, with each diffusion solve D^{-1}
    # replaced by the degree-m Chebyshev approximant r(d) = (1 - T_{m+1}((th - d)/de)
    # / T_{m+1}(th/de)) / d on D's interval [sD, sD + sqrt(kt) max kK]:
    #   b2' = r (b2 - kt g b1),  chi2 = r b2',  chi1 = b1 + (b2' - sD chi2) / sqrt(kt).
    ks, shape, h = _case_grid(lat)
    _, c = _paper_P_symbol(ks[j], dt, p, shape, h, "fold")
    lmin, lmax = c["sD"], c["sD"] + c["mu"] * sum(4.0 / (hd * hd) for hd in h)
    th, de = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
    T = np.polynomial.chebyshev.Chebyshev.basis(m + 1)
    r = (1.0 - T((th - c["dq"]) / de) / T(th / de)) / c["dq"]
    want = np.empty(shape + (2, 2), dtype=complex)
    for b, (b1, b2) in enumerate(((1.0, 0.0), (0.0, 1.0))):
        b2p = r * (b2 - c["kt"] * c["g"] * b1)
        chi2 = r * b2p
        want[..., 0, b] = b1 + (b2p - c["sD"] * chi2) / c["mu"]
        want[..., 1, b] = chi2
    got = _block_symbol(lambda a, b: O.apply_Pinv(a, b, ks[j], dt, p, h, m, "fold"), shape)
    np.testing.assert_allclose(got, want, atol=1e-12 * np.abs(want).max())


@pytest.mark.parametrize(
    "j,tau_mode,lo,hi",
    [(0, "plain", 0.1252, 1.956), (2, "plain", 0.1252, 1.956), (1, "plain", 0.166, 1.694),
     (0, "fold", 0.1244, 1.935), (2, "fold", 0.1244, 1.935)],
)
def test_discrete_preconditioned_spectrum(j, tau_mode, lo, hi):
    # Discrete counterpart of the paper's spectrum analysis (Sec. II.B): the
    # eigenvalues of A_j(q) P_j(q)^{-1} for the hex k_j at h = pi/2, dt = 1,
    # exact inner solves, over the frequencies of a 128^2 grid.  The interval
    # ends are those of the 2x2 symbols of the discrete operators over the whole
    # Brillouin zone (P(q) as in Eq. preconditioner, A(q) = [[1, -g], [kt g, a]]),
    # rounded to 4 digits; the spectrum is real and positive.
    k = O.hex_k()[j]
    shape, h, dt = (128, 128), H2, 1.0
    A = _block_symbol(lambda a, b: O.apply_A(a, b, k, dt, P, h), shape)
    Pinv = _block_symbol(lambda a, b: O.apply_Pinv(a, b, k, dt, P, h, None, tau_mode), shape)
    ev = np.linalg.eigvals(A @ Pinv)
    assert np.abs(ev.imag).max() < 1e-9
    assert ev.real.min() == pytest.approx(lo, abs=5e-4)
    assert ev.real.max() == pytest.approx(hi, abs=5e-4)
